// Design-update kernels of the optimization loop (Sec. 3.2): the ascent step
// on rho, the grayness measure zeta = 4 rho~^T (1 - rho~) / M of the filtered
// design, and the final thresholding.
#include "fdtd_internal.h"

namespace fdtd {

namespace {

constexpr int TPB = 256;
inline int blocks_for(long long n, int cap = 152 * 8)
{
    long long b = (n + TPB - 1) / TPB;
    return (int)(b < 1 ? 1 : (b < cap ? b : cap));
}

__device__ __forceinline__ double warp_max(double v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// out[0] = max |g| (non-negative doubles order like their bit patterns, so an
// integer atomicMax on the bits is exact).  out[0] must start at 0.
__global__ void k_absmax(const double *g, long long n, unsigned long long *out)
{
    double m = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        m = fmax(m, fabs(g[k]));  // fmax drops NaN
    m = warp_max(m);
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// rho <- clip(rho + move * g / max|g|, 0, 1); unchanged where max|g| = 0.
template <typename R>
__global__ void k_ascent(R *rho, const double *g, long long n, double move, const unsigned long long *gmax)
{
    const double m = __longlong_as_double((long long)*gmax);
    if (!(m > 0.0)) return;
    const double s = move / m;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const double v = (double)rho[k] + s * g[k];
        rho[k] = (R)fmin(1.0, fmax(0.0, v));
    }
}

// Sum over the design box of rho~ (1 - rho~), gap nodes excluded; pitched
// layout (rows of dp, box at column off), rows = dny (times dnz in 3D),
// row width dnx.  Accumulates into *acc (FP64).
template <typename R>
__global__ void k_gray(const R *rt, long long rows, int dnx, int dp, int off, int rows_per_plane, int gx0, int gy0,
                       int gz0, int gnx, int gny, int gnz, double *acc)
{
    double s = 0.0;
    const long long n = rows * dnx;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(k % dnx);
        const long long r = k / dnx;
        const int y = (int)(r % rows_per_plane), z = (int)(r / rows_per_plane);
        const bool gap = (unsigned)(x - gx0) < (unsigned)gnx && (unsigned)(y - gy0) < (unsigned)gny &&
                         (unsigned)(z - gz0) < (unsigned)gnz;
        if (gap) continue;
        const double v = (double)rt[r * dp + off + x];
        s += v * (1.0 - v);
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) atomicAdd(acc, s);
}

__global__ void k_scale1(double *x, double s) { *x *= s; }

template <typename R>
__global__ void k_threshold(R *rho, long long n, double level)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        rho[k] = (double)rho[k] >= level ? R(1) : R(0);
}

}  // namespace

template <typename R>
void launch_ascent(R *rho, const double *g, long long n, double move, unsigned long long *gmax, cudaStream_t st)
{
    launch_zero_bytes(gmax, sizeof(unsigned long long), st);
    k_absmax<<<blocks_for(n), TPB, 0, st>>>(g, n, gmax);
    k_ascent<R><<<blocks_for(n), TPB, 0, st>>>(rho, g, n, move, gmax);
}

template <typename R>
void launch_grayness(const R *rt, long long rows, int dnx, int dp, int off, int rows_per_plane, int gx0, int gy0,
                     int gz0, int gnx, int gny, int gnz, double *acc, cudaStream_t st)
{
    launch_zero_bytes(acc, sizeof(double), st);
    k_gray<R><<<blocks_for(rows * dnx), TPB, 0, st>>>(rt, rows, dnx, dp, off, rows_per_plane, gx0, gy0, gz0, gnx, gny,
                                                       gnz, acc);
}

void launch_scale1(double *x, double s, cudaStream_t st) { k_scale1<<<1, 1, 0, st>>>(x, s); }

template <typename R>
void launch_threshold(R *rho, long long n, double level, cudaStream_t st)
{
    k_threshold<R><<<blocks_for(n), TPB, 0, st>>>(rho, n, level);
}

template void launch_ascent<float>(float *, const double *, long long, double, unsigned long long *, cudaStream_t);
template void launch_ascent<double>(double *, const double *, long long, double, unsigned long long *, cudaStream_t);
template void launch_grayness<float>(const float *, long long, int, int, int, int, int, int, int, int, int, int,
                                     double *, cudaStream_t);
template void launch_grayness<double>(const double *, long long, int, int, int, int, int, int, int, int, int, int,
                                      double *, cudaStream_t);
template void launch_threshold<float>(float *, long long, double, cudaStream_t);
template void launch_threshold<double>(double *, long long, double, cudaStream_t);

}  // namespace fdtd
