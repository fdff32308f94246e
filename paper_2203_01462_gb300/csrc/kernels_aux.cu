// Auxiliary kernels: design upload and range check, the Gaussian design
// filter and its transpose (Eq. 26, 27), the objective reduction (Eq. 24),
// gradient assembly, and plain copies for checkpoints.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fdtd_internal.h"

namespace fdtd {

namespace {

constexpr int TPB = 256;

inline int blocks_for(long long n, int per_block = TPB, int cap = 152 * 16)
{
    long long b = (n + per_block - 1) / per_block;
    if (b < 1) b = 1;
    return (int)(b < cap ? b : cap);
}

template <typename R>
__global__ void k_copy_check_rho(const R *src, R *dst, long long n, unsigned *err)
{
    bool bad = false;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const R v = src[k];
        bad |= !(v >= R(0) && v <= R(1));  // also catches NaN
        dst[k] = v;
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(err, ERR_RANGE);
}

// Stability guard: flag a state word that is not finite or exceeds `bound`
// in magnitude.  Sets ERR_UNSTABLE in the device error word and, when
// `host_flag` (a mapped host word) is given, writes `tag` there so that the
// host loop that enqueues the steps can stop early.  Reads only.
template <typename R>
__global__ void k_guard(const R *state, long long n, R bound, unsigned *err, unsigned *host_flag, unsigned tag)
{
    bool bad = false;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x)
        bad |= !(fabs(state[k]) <= bound);  // also catches NaN
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) {
        atomicOr(err, ERR_UNSTABLE);
        if (host_flag) {
            *(volatile unsigned *)host_flag = tag;
            __threadfence_system();
        }
    }
}

// One separable pass of the normalised Gaussian filter along x (rows) or y
// (columns) of a w x h design array.  Forward:  out[i] = inv_norm[i] *
// sum_k wts[k] in[i + k].  Transpose: out[i] = sum_k wts[k] inv_norm[i + k]
// in[i + k] (the weights are symmetric).  Taps leaving the box are dropped.
template <typename T>
__global__ void k_filter_rows(const T *in, T *out, int w, int h, int R_, const T *wts, const T *inv_norm,
                              int transpose)
{
    const long long n = (long long)w * h;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(k % w);
        const T *row = in + (k - x);
        T acc = T(0);
        for (int t = -R_; t <= R_; ++t) {
            const int xx = x + t;
            if (xx < 0 || xx >= w) continue;
            acc += transpose ? wts[t + R_] * inv_norm[xx] * row[xx] : wts[t + R_] * row[xx];
        }
        out[k] = transpose ? acc : acc * inv_norm[x];
    }
}

template <typename T>
__global__ void k_filter_cols(const T *in, T *out, int w, int h, int R_, const T *wts, const T *inv_norm,
                              int transpose)
{
    const long long n = (long long)w * h;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(k % w);
        const int y = (int)(k / w);
        T acc = T(0);
        for (int t = -R_; t <= R_; ++t) {
            const int yy = y + t;
            if (yy < 0 || yy >= h) continue;
            const T v = in[(long long)yy * w + x];
            acc += transpose ? wts[t + R_] * inv_norm[yy] * v : wts[t + R_] * v;
        }
        out[k] = transpose ? acc : acc * inv_norm[y];
    }
}

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// W~ = coef * sum of squares of the recorded gap field (Eq. 24), FP64
// accumulation, one block (the history is a few hundred kB at most).
template <typename R>
__global__ void __launch_bounds__(256) k_objective_part(const R *h, long long count, double *part)
{
    __shared__ double sh[8];
    double acc = 0.0;
    for (long long k = blockIdx.x * 256LL + threadIdx.x; k < count; k += (long long)gridDim.x * 256) {
        const double v = (double)h[k];
        acc += v * v;
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < 8 ? sh[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) part[blockIdx.x] = v;
    }
}

// W = coef * (sum of the block partials, in a fixed order).
__global__ void __launch_bounds__(256) k_objective_final(const double *part, int nb, double coef, double *W,
                                                         double *W_user, unsigned *err)
{
    __shared__ double sh[8];
    double acc = 0.0;
    for (int k = threadIdx.x; k < nb; k += 256) acc += part[k];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < 8 ? sh[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) {
            const double w = coef * v;
            *W = w;
            if (W_user) *W_user = w;
            if (!isfinite(w)) atomicOr(err, ERR_NONFINITE);
        }
    }
}

__global__ void k_assemble_2d(const double *G, double *out, int dnx, int dny, int off, int dp, int gx0, int gy0,
                              int gnx, int gny, double scale)
{
    const long long n = (long long)dnx * dny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(k % dnx), y = (int)(k / dnx);
        const bool gap = (unsigned)(x - gx0) < (unsigned)gnx && (unsigned)(y - gy0) < (unsigned)gny;
        out[k] = gap ? 0.0 : scale * G[(long long)y * dp + off + x];
    }
}

// 3D: out (compact dx x dy x dz) = scale * G (pitched rows of dp from column
// off), zero inside the gap box (relative to the design box).
__global__ void k_assemble_3d(const double *G, double *out, int dx, int dy, int dz, int off, int dp, int gx0, int gy0,
                              int gz0, int gnx, int gny, int gnz, double scale)
{
    const long long n = (long long)dx * dy * dz;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(k % dx);
        const long long r = k / dx;  // row index (y + z * dy)
        const int y = (int)(r % dy), z = (int)(r / dy);
        const bool gap = (unsigned)(x - gx0) < (unsigned)gnx && (unsigned)(y - gy0) < (unsigned)gny &&
                         (unsigned)(z - gz0) < (unsigned)gnz;
        out[k] = gap ? 0.0 : scale * G[r * dp + off + x];
    }
}

template <typename T>
__global__ void k_pitch2d(const T *compact, T *pitched, int dnx, int dny, int off, int dp)
{
    const long long n = (long long)dp * dny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int xp = (int)(k % dp), y = (int)(k / dp);
        const int x = xp - off;
        pitched[k] = (x >= 0 && x < dnx) ? compact[(long long)y * dnx + x] : T(0);
    }
}

__global__ void k_zero_gap_2d(double *g, int dnx, int gx0, int gy0, int gnx, int gny)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= gnx * gny) return;
    const int x = gx0 + k % gnx, y = gy0 + k / gnx;
    g[(long long)y * dnx + x] = 0.0;
}

template <typename R>
__global__ void k_to_double(const R *in, double *out, long long n)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x)
        out[k] = (double)in[k];
}

// 16-byte vector copy / clear; sizes are multiples of 256 bytes by
// construction of the workspace layout, tails handled bytewise anyway.
__global__ void k_copy_bytes(const uint4 *src, uint4 *dst, size_t n16, const unsigned char *s8,
                             unsigned char *d8, size_t tail_from, size_t bytes)
{
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n16; k += (size_t)gridDim.x * blockDim.x)
        dst[k] = src[k];
    for (size_t k = tail_from + blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < bytes;
         k += (size_t)gridDim.x * blockDim.x)
        d8[k] = s8[k];
}

__global__ void k_zero_bytes(uint4 *dst, size_t n16, unsigned char *d8, size_t tail_from, size_t bytes)
{
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n16; k += (size_t)gridDim.x * blockDim.x)
        dst[k] = make_uint4(0, 0, 0, 0);
    for (size_t k = tail_from + blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < bytes;
         k += (size_t)gridDim.x * blockDim.x)
        d8[k] = 0;
}

// 16-bit checkpoint of a state block: slabs of SLAB consecutive words, one
// warp per slab.  The warp finds max |x| (shuffle reduction), picks a scale
// (FP16: the maximum maps to 2^15, keeping small values out of the subnormal
// range; BF16: the maximum maps to 1) and stores x * scale.  Restoring
// divides by the scale.
template <typename T> __device__ __forceinline__ T to16(float v);
template <> __device__ __forceinline__ __half to16<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 to16<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
__device__ __forceinline__ float from16(__half v) { return __half2float(v); }
__device__ __forceinline__ float from16(__nv_bfloat16 v) { return __bfloat162float(v); }
template <typename T> __device__ __forceinline__ float target_max();
template <> __device__ __forceinline__ float target_max<__half>() { return 32768.0f; }
template <> __device__ __forceinline__ float target_max<__nv_bfloat16>() { return 1.0f; }

template <typename R, typename T>
__global__ void k_snap_pack(const R *src, T *dst, float *scales, long long n)
{
    const long long nslab = (n + SNAP_SLAB - 1) / SNAP_SLAB;
    const int lane = threadIdx.x & 31;
    for (long long sl = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; sl < nslab;
         sl += ((long long)gridDim.x * blockDim.x) >> 5) {
        const long long b = sl * SNAP_SLAB, e = min(b + SNAP_SLAB, n);
        float m = 0.0f;
        for (long long k = b + lane; k < e; k += 32) m = fmaxf(m, fabsf((float)src[k]));
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        // A slab whose largest word is below 1e-30 keeps scale 1 (its words
        // round to zero) so that the scale cannot overflow.
        const float sc = m > 1e-30f ? target_max<T>() / m : 1.0f;
        if (lane == 0) scales[sl] = sc;
        for (long long k = b + lane; k < e; k += 32) dst[k] = to16<T>((float)src[k] * sc);
    }
}

template <typename R, typename T>
__global__ void k_snap_unpack(const T *src, const float *scales, R *dst, long long n)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x)
        dst[k] = (R)(from16(src[k]) / scales[k / SNAP_SLAB]);
}

}  // namespace

template <typename R>
void launch_snap_pack(int kind, const R *src, void *dst, float *scales, long long n, cudaStream_t st)
{
    const int blocks = blocks_for(((n + SNAP_SLAB - 1) / SNAP_SLAB) * 32);
    if (kind == 2) k_snap_pack<R, __half><<<blocks, TPB, 0, st>>>(src, (__half *)dst, scales, n);
    else k_snap_pack<R, __nv_bfloat16><<<blocks, TPB, 0, st>>>(src, (__nv_bfloat16 *)dst, scales, n);
}

template <typename R>
void launch_snap_unpack(int kind, const void *src, const float *scales, R *dst, long long n, cudaStream_t st)
{
    if (kind == 2) k_snap_unpack<R, __half><<<blocks_for(n), TPB, 0, st>>>((const __half *)src, scales, dst, n);
    else k_snap_unpack<R, __nv_bfloat16><<<blocks_for(n), TPB, 0, st>>>((const __nv_bfloat16 *)src, scales, dst, n);
}

template void launch_snap_pack<float>(int, const float *, void *, float *, long long, cudaStream_t);
template void launch_snap_pack<double>(int, const double *, void *, float *, long long, cudaStream_t);
template void launch_snap_unpack<float>(int, const void *, const float *, float *, long long, cudaStream_t);
template void launch_snap_unpack<double>(int, const void *, const float *, double *, long long, cudaStream_t);

template <typename R>
void launch_copy_check_rho(const R *src, R *dst, long long n, unsigned *err, cudaStream_t st)
{
    k_copy_check_rho<R><<<blocks_for(n), TPB, 0, st>>>(src, dst, n, err);
}

template <typename R>
void launch_guard(const R *state, long long n, double bound, unsigned *err, unsigned *host_flag, unsigned tag,
                  cudaStream_t st)
{
    k_guard<R><<<blocks_for(n, TPB, 152 * 8), TPB, 0, st>>>(state, n, (R)bound, err, host_flag, tag);
}
template void launch_guard<float>(const float *, long long, double, unsigned *, unsigned *, unsigned, cudaStream_t);
template void launch_guard<double>(const double *, long long, double, unsigned *, unsigned *, unsigned,
                                   cudaStream_t);

template <typename T>
void launch_filter_rows(const T *in, T *out, int w, int h, int R_, const T *wts, const T *inv_norm,
                        int transpose, cudaStream_t st)
{
    k_filter_rows<T><<<blocks_for((long long)w * h), TPB, 0, st>>>(in, out, w, h, R_, wts, inv_norm, transpose);
}

template <typename T>
void launch_filter_cols(const T *in, T *out, int w, int h, int R_, const T *wts, const T *inv_norm,
                        int transpose, cudaStream_t st)
{
    k_filter_cols<T><<<blocks_for((long long)w * h), TPB, 0, st>>>(in, out, w, h, R_, wts, inv_norm, transpose);
}

// W~ of Eq. (24) from the recorded gap history: block partial sums of E^2
// in FP64 (the grid size depends only on count, so the sum is
// deterministic), then one block adds them in order and scales by coef.
template <typename R>
void launch_objective(const R *gap_hist, long long count, double coef, double *W, double *W_user, double *part,
                      unsigned *err, cudaStream_t st)
{
    long long nb = (count + 4 * 256 - 1) / (4 * 256);
    nb = nb < 1 ? 1 : (nb > OBJ_BLOCKS ? OBJ_BLOCKS : nb);
    k_objective_part<R><<<(int)nb, 256, 0, st>>>(gap_hist, count, part);
    k_objective_final<<<1, 256, 0, st>>>(part, (int)nb, coef, W, W_user, err);
}

void launch_assemble_2d(const double *G, double *out, int dnx, int dny, int off, int dp, int gx0, int gy0,
                        int gnx, int gny, double scale, cudaStream_t st)
{
    k_assemble_2d<<<blocks_for((long long)dnx * dny), TPB, 0, st>>>(G, out, dnx, dny, off, dp, gx0, gy0, gnx, gny,
                                                                   scale);
}

void launch_assemble_3d(const double *G, double *out, int dx, int dy, int dz, int off, int dp, int gx0, int gy0,
                        int gz0, int gnx, int gny, int gnz, double scale, cudaStream_t st)
{
    k_assemble_3d<<<blocks_for((long long)dx * dy * dz), TPB, 0, st>>>(G, out, dx, dy, dz, off, dp, gx0, gy0, gz0,
                                                                       gnx, gny, gnz, scale);
}

template <typename T>
void launch_pitch2d(const T *compact, T *pitched, int dnx, int dny, int off, int dp, cudaStream_t st)
{
    k_pitch2d<T><<<blocks_for((long long)dp * dny), TPB, 0, st>>>(compact, pitched, dnx, dny, off, dp);
}

void launch_zero_gap_2d(double *g, int dnx, int gx0, int gy0, int gnx, int gny, cudaStream_t st)
{
    const int n = gnx * gny;
    if (n <= 0) return;
    k_zero_gap_2d<<<(n + TPB - 1) / TPB, TPB, 0, st>>>(g, dnx, gx0, gy0, gnx, gny);
}

// Discrete Fourier transform of a recorded time series (nt steps of m
// entries, x[n * m + e]) at nf frequencies, one thread per (frequency,
// entry):  out[2 (f m + e) + 0/1] = dt sum_n x[n m + e] (cos, -sin)(w n),
// w = 2 pi freq[f] dt.  The phase factor advances by one complex rotation
// per step and is re-seeded from sincos every 256 steps, so its rounding
// error stays at a few ulp.
template <typename R>
__global__ void k_gap_dft(const R *x, long long nt, int m, double dt, const double *freqs, int nf, double *out)
{
    const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (id >= (long long)nf * m) return;
    const int f = (int)(id / m), e = (int)(id % m);
    const double w = 2.0 * 3.14159265358979323846 * freqs[f] * dt;
    double sw, cw;
    sincos(w, &sw, &cw);
    double re = 0.0, im = 0.0;
    for (long long n0 = 0; n0 < nt; n0 += 256) {
        double zs, zc;
        sincos(w * (double)n0, &zs, &zc);
        double zr = zc, zi = -zs;  // e^{-i w n}
        const long long n1 = n0 + 256 < nt ? n0 + 256 : nt;
        for (long long n = n0; n < n1; ++n) {
            const double v = (double)x[n * m + e];
            re += v * zr;
            im += v * zi;
            const double t = zr * cw + zi * sw;  // times e^{-i w}
            zi = zi * cw - zr * sw;
            zr = t;
        }
    }
    out[2 * id] = re * dt;
    out[2 * id + 1] = im * dt;
}

template <typename R>
void launch_gap_dft(const R *x, long long nt, int m, double dt, const double *freqs, int nf, double *out,
                    cudaStream_t st)
{
    const long long n = (long long)nf * m;
    k_gap_dft<R><<<(unsigned)((n + TPB - 1) / TPB), TPB, 0, st>>>(x, nt, m, dt, freqs, nf, out);
}

template <typename R>
void launch_to_double(const R *in, double *out, long long n, cudaStream_t st)
{
    k_to_double<R><<<blocks_for(n), TPB, 0, st>>>(in, out, n);
}

void launch_copy_bytes(const void *src, void *dst, size_t bytes, cudaStream_t st)
{
    if (!bytes) return;
    const size_t n16 = bytes / 16;
    k_copy_bytes<<<blocks_for((long long)(n16 ? n16 : 1)), TPB, 0, st>>>(
        (const uint4 *)src, (uint4 *)dst, n16, (const unsigned char *)src, (unsigned char *)dst, n16 * 16, bytes);
}

void launch_zero_bytes(void *dst, size_t bytes, cudaStream_t st)
{
    if (!bytes) return;
    const size_t n16 = bytes / 16;
    k_zero_bytes<<<blocks_for((long long)(n16 ? n16 : 1)), TPB, 0, st>>>((uint4 *)dst, n16, (unsigned char *)dst,
                                                                          n16 * 16, bytes);
}

template void launch_copy_check_rho<float>(const float *, float *, long long, unsigned *, cudaStream_t);
template void launch_copy_check_rho<double>(const double *, double *, long long, unsigned *, cudaStream_t);
template void launch_filter_rows<float>(const float *, float *, int, int, int, const float *, const float *, int,
                                        cudaStream_t);
template void launch_filter_rows<double>(const double *, double *, int, int, int, const double *, const double *,
                                         int, cudaStream_t);
template void launch_filter_cols<float>(const float *, float *, int, int, int, const float *, const float *, int,
                                        cudaStream_t);
template void launch_filter_cols<double>(const double *, double *, int, int, int, const double *, const double *,
                                         int, cudaStream_t);
template void launch_objective<float>(const float *, long long, double, double *, double *, double *,
                                      unsigned *, cudaStream_t);
template void launch_objective<double>(const double *, long long, double, double *, double *, double *,
                                       unsigned *, cudaStream_t);
template void launch_pitch2d<float>(const float *, float *, int, int, int, int, cudaStream_t);
template void launch_pitch2d<double>(const double *, double *, int, int, int, int, cudaStream_t);
template void launch_gap_dft<float>(const float *, long long, int, double, const double *, int, double *,
                                    cudaStream_t);
template void launch_gap_dft<double>(const double *, long long, int, double, const double *, int, double *,
                                     cudaStream_t);
template void launch_to_double<float>(const float *, double *, long long, cudaStream_t);
template void launch_to_double<double>(const double *, double *, long long, cudaStream_t);

}  // namespace fdtd
