// Design-update kernels of the optimization loop (Sec. 3.2): the ascent step
// on rho, the method of moving asymptotes with the conservative inner loop of
// GCMMA, the grayness measure zeta = 4 rho~^T (1 - rho~) / M of the filtered
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

// Two FP64 sums per block, reduced by shuffles and shared memory, written
// to part[2 * block + 0/1]; k_sum_partials then adds the blocks in a fixed
// order, so the totals do not depend on scheduling.
__device__ __forceinline__ void block_sum2(double a, double b, double *part)
{
    __shared__ double sh[2][TPB / 32];
    a = warp_sum(a);
    b = warp_sum(b);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { sh[0][w] = a; sh[1][w] = b; }
    __syncthreads();
    if (w == 0) {
        a = l < TPB / 32 ? sh[0][l] : 0.0;
        b = l < TPB / 32 ? sh[1][l] : 0.0;
        a = warp_sum(a);
        b = warp_sum(b);
        if (l == 0) { part[2 * blockIdx.x] = a; part[2 * blockIdx.x + 1] = b; }
    }
}

// One warp: sums[c] = sum over blocks of part[2 * block + c], c = 0, 1.
__global__ void k_sum_partials(const double *part, int nblocks, double *sums)
{
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += 32) {
        a += part[2 * i];
        b += part[2 * i + 1];
    }
    a = warp_sum(a);
    b = warp_sum(b);
    if (threadIdx.x == 0) { sums[0] = a; sums[1] = b; }
}

// Method of moving asymptotes (Svanberg, IJNME 1987) for max W~ over the box
// [0, 1]^M, written as min f with f = -s W~.  State: four FP64 arrays of n
// entries, back to back: x^{k-1} (x^k once this kernel has run), x^{k-2},
// L, U.  Iteration k sets the asymptotes from the last three iterates:
// distance 0.5 for k < 2, else the previous distance times 0.7 where the
// coordinate oscillates, 1.2 where it moves monotonically, 1 where it
// stalled, kept within [0.01, 10].  Also sums |g| (for the initial GCMMA
// rho0) and the squared first-order optimality residual (g with the entries
// removed where a bound is active and g points out of the box).
template <typename R>
__global__ void __launch_bounds__(TPB) k_mma_asymptotes(const R *rho, const double *g, double *st, long long n, int k,
                                                        double *part)
{
    double *x1 = st, *x2 = st + n, *lo = st + 2 * n, *up = st + 3 * n;
    double sa = 0.0, sr = 0.0;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
        const double x = (double)rho[j];
        double L, U;
        if (k < 2) {
            L = x - 0.5;
            U = x + 0.5;
        } else {
            const double a = x1[j], t = (x - a) * (a - x2[j]);
            const double fac = t < 0.0 ? 0.7 : (t > 0.0 ? 1.2 : 1.0);
            L = fmin(fmax(x - fac * (a - lo[j]), x - 10.0), x - 0.01);
            U = fmin(fmax(x + fac * (up[j] - a), x + 0.01), x + 10.0);
        }
        x2[j] = x1[j];
        x1[j] = x;
        lo[j] = L;
        up[j] = U;
        const double gj = g[j];
        sa += fabs(gj);
        if (!((x <= 0.0 && gj < 0.0) || (x >= 1.0 && gj > 0.0))) sr += gj * gj;
    }
    block_sum2(sa, sr, part);
}

// The MMA subproblem with the GCMMA term raa0 (Svanberg, SIAM J. Optim.
// 2002): with df = -s g,
//   p = (U-x)^2 (1.001 max(df,0) + 0.001 max(-df,0) + raa0),
//   q = (x-L)^2 (0.001 max(df,0) + 1.001 max(-df,0) + raa0),
// each coordinate's minimiser of p/(U-y) + q/(y-L) is
// (sqrt(p) L + sqrt(q) U)/(sqrt(p) + sqrt(q)), clipped to
// alpha = max(0, L + 0.1 (x-L), x - move), beta = min(1, U - 0.1 (U-x), x + move).
// Entries with g = 0 (gap nodes) stay at x.  Writes y in the field
// precision and sums, with y as stored, the approximation change
// f~(y) - f(x) and the GCMMA term d(y) = sum (U-L)(y-x)^2/((U-y)(y-L)).
template <typename R>
__global__ void __launch_bounds__(TPB) k_mma_solve(const double *st, const double *g, long long n, double s,
                                                   double raa0, double move, R *out, double *part)
{
    const double *xk = st, *lo = st + 2 * n, *up = st + 3 * n;
    double sa = 0.0, sd = 0.0;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
        const double x = xk[j], gj = g[j];
        if (gj == 0.0) {
            out[j] = (R)x;
            continue;
        }
        const double L = lo[j], U = up[j], df = -s * gj;
        const double pos = fmax(df, 0.0), neg = fmax(-df, 0.0);
        const double p = (U - x) * (U - x) * (1.001 * pos + 0.001 * neg + raa0);
        const double q = (x - L) * (x - L) * (0.001 * pos + 1.001 * neg + raa0);
        const double alpha = fmax(fmax(0.0, L + 0.1 * (x - L)), x - move);
        const double beta = fmin(fmin(1.0, U - 0.1 * (U - x)), x + move);
        const double sp = sqrt(p), sq = sqrt(q);
        const double y = fmin(fmax((sp * L + sq * U) / (sp + sq), alpha), beta);
        const R yr = (R)y;
        const double yd = (double)yr;
        out[j] = yr;
        sa += p * (yd - x) / ((U - yd) * (U - x)) + q * (x - yd) / ((yd - L) * (x - L));
        sd += (U - L) * (yd - x) * (yd - x) / ((U - yd) * (yd - L));
    }
    block_sum2(sa, sd, part);
}

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
                     int gz0, int gnx, int gny, int gnz, double *acc, cudaStream_t st, bool accumulate)
{
    if (!accumulate) launch_zero_bytes(acc, sizeof(double), st);
    k_gray<R><<<blocks_for(rows * dnx), TPB, 0, st>>>(rt, rows, dnx, dp, off, rows_per_plane, gx0, gy0, gz0, gnx, gny,
                                                       gnz, acc);
}

void launch_scale1(double *x, double s, cudaStream_t st) { k_scale1<<<1, 1, 0, st>>>(x, s); }

template <typename R>
void launch_mma_asymptotes(const R *rho, const double *g, double *state, long long n, int k, double *part,
                           double *sums, cudaStream_t st)
{
    const int nb = blocks_for(n, MMA_BLOCKS);
    k_mma_asymptotes<R><<<nb, TPB, 0, st>>>(rho, g, state, n, k, part);
    k_sum_partials<<<1, 32, 0, st>>>(part, nb, sums);
}

template <typename R>
void launch_mma_solve(const double *state, const double *g, long long n, double s, double raa0, double move, R *out,
                      double *part, double *sums, cudaStream_t st)
{
    const int nb = blocks_for(n, MMA_BLOCKS);
    k_mma_solve<R><<<nb, TPB, 0, st>>>(state, g, n, s, raa0, move, out, part);
    k_sum_partials<<<1, 32, 0, st>>>(part, nb, sums);
}

// Mirror average over the design layout: each entry and its image across the
// mid-plane of its rectangle normal to `axis` both become their mean.  The
// layout is one or two rectangles (x fastest); only the lower index of each
// pair writes, so pairs never race.
template <typename T>
__global__ void k_mirror_avg(T *v, DesignRects r, int axis)
{
    long long total = 0;
    for (int q = 0; q < r.n; ++q) total += (long long)r.w[q] * r.h[q] * r.d[q];
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        int q = 0;
        long long k = t;
        while (q + 1 < r.n && k >= (long long)r.w[q] * r.h[q] * r.d[q]) {
            k -= (long long)r.w[q] * r.h[q] * r.d[q];
            ++q;
        }
        const int w = r.w[q], h = r.h[q], d = r.d[q];
        int x = (int)(k % w), y = (int)((k / w) % h), z = (int)(k / ((long long)w * h));
        if (axis == 0) x = w - 1 - x;
        else if (axis == 1) y = h - 1 - y;
        else z = d - 1 - z;
        const long long km = ((long long)z * h + y) * w + x;
        if (km <= k) continue;
        T *base = v + r.off[q];
        const double m = 0.5 * ((double)base[k] + (double)base[km]);
        base[k] = (T)m;
        base[km] = (T)m;
    }
}

// Fixed design variables: rho = value and gradient 0 where mask is set.
template <typename T>
__global__ void k_fix(T *rho, double *g, const unsigned char *mask, long long n, double value)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        if (mask[k]) {
            if (rho) rho[k] = (T)value;
            if (g) g[k] = 0.0;
        }
}

template <typename T>
void launch_mirror_avg(T *v, const DesignRects &r, int axis, cudaStream_t st)
{
    long long total = 0;
    for (int q = 0; q < r.n; ++q) total += (long long)r.w[q] * r.h[q] * r.d[q];
    k_mirror_avg<T><<<blocks_for(total), TPB, 0, st>>>(v, r, axis);
}

template <typename T>
void launch_fix(T *rho, double *g, const unsigned char *mask, long long n, double value, cudaStream_t st)
{
    k_fix<T><<<blocks_for(n), TPB, 0, st>>>(rho, g, mask, n, value);
}

template void launch_mirror_avg<float>(float *, const DesignRects &, int, cudaStream_t);
template void launch_mirror_avg<double>(double *, const DesignRects &, int, cudaStream_t);
template void launch_fix<float>(float *, double *, const unsigned char *, long long, double, cudaStream_t);
template void launch_fix<double>(double *, double *, const unsigned char *, long long, double, cudaStream_t);

template <typename R>
void launch_threshold(R *rho, long long n, double level, cudaStream_t st)
{
    k_threshold<R><<<blocks_for(n), TPB, 0, st>>>(rho, n, level);
}

template void launch_ascent<float>(float *, const double *, long long, double, unsigned long long *, cudaStream_t);
template void launch_ascent<double>(double *, const double *, long long, double, unsigned long long *, cudaStream_t);
template void launch_grayness<float>(const float *, long long, int, int, int, int, int, int, int, int, int, int,
                                     double *, cudaStream_t, bool);
template void launch_grayness<double>(const double *, long long, int, int, int, int, int, int, int, int, int, int,
                                      double *, cudaStream_t, bool);
template void launch_mma_asymptotes<float>(const float *, const double *, double *, long long, int, double *,
                                           double *, cudaStream_t);
template void launch_mma_asymptotes<double>(const double *, const double *, double *, long long, int, double *,
                                            double *, cudaStream_t);
template void launch_mma_solve<float>(const double *, const double *, long long, double, double, double, float *,
                                      double *, double *, cudaStream_t);
template void launch_mma_solve<double>(const double *, const double *, long long, double, double, double, double *,
                                       double *, double *, cudaStream_t);
template void launch_threshold<float>(float *, long long, double, cudaStream_t);
template void launch_threshold<double>(double *, long long, double, cudaStream_t);

}  // namespace fdtd
