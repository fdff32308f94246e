// 2D leapfrog with E in plane (Ex, Ey, Hz + Drude Jx, Jy + CPML) for sm_103a:
// the paper's 2D "TM" polarisation, in which surface plasmons exist.
//
// Ex(i, j) lives on the edge (i+1/2, j), Ey(i, j) on (i, j+1/2), Hz(i, j) at
// the cell centre (i+1/2, j+1/2).  Two launches per step, each in place:
//   H:  mu0 dHz/dt = -(dEy/dx - dEx/dy)         (forward differences)
//   E:  Eq. (10a,b) per edge with curl_x = dHz/dy, curl_y = -dHz/dx
//       (backward differences), J and sigma E averaged over the step.
// Tangential E vanishes on the walls (Ex on the rows j = 0, ny-1; Ey on the
// columns i = 0, nx-1).  Each derivative takes its CPML term inside the slab
// of its axis.  Every design edge takes the material of its own density
// (Eq. 5); the adjoint accumulates the Eq. (25) bracket per edge in FP64.
//
// One thread per (i, j), 32 x 4 threads per block (a sweep of 32 x 2 / 4 / 8 /
// 16 on the paper geometry: 32 x 4 fastest, by 5 %): a warp reads 32
// consecutive entries of a row of each array.

#include "coef_slots.cuh"
#include "fdtd_internal.h"
#include "launch.cuh"

namespace fdtd {

namespace {

constexpr int BX = 32, BY = 4;

__device__ __forceinline__ bool in_range(int v, int lo, int n) { return (unsigned)(v - lo) < (unsigned)n; }
__device__ __forceinline__ void wait_previous_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp(double x) { return __drcp_rn(x); }

// Slab index of a position (E: node p, H: half position p + 1/2) along an
// axis of n nodes, or -1 outside the absorbing layer.
__device__ __forceinline__ int slabE(int p, int n, int np) { return p < np ? p : (p >= n - np ? p - (n - 2 * np) : -1); }
__device__ __forceinline__ int slabH(int p, int n, int np)
{
    return p < np ? p : ((p >= n - 1 - np && p < n - 1) ? np + p - (n - 1 - np) : -1);
}

// H half step of the cell (i, j) (Hz exists on the (nx-1) x (ny-1) cells).
template <typename R>
__device__ __forceinline__ void h_cell(const GeoP &g, const StateP<R> &s, const Coef<R> &c, const PmlP<R> &pm, int i,
                                       int j)
{
    if (i > g.nx - 2 || j > g.ny - 2) return;
    const long long q = (long long)j * g.px + i;
    const R dEy = s.Ey[q + 1] - s.Ey[q];     // d_x Ey
    const R dEx = s.Ex[q + g.px] - s.Ex[q];  // d_y Ex
    R tx = dEy * __ldg(pm.kiH[0] + i), ty = dEx * __ldg(pm.kiH[1] + j);
    const int np = g.npml;
    const int sx = slabH(i, g.nx, np), sy = slabH(j, g.ny, np);
    if (sx >= 0) {
        R &p = s.phzx[(long long)j * 2 * np + sx];
        p = __ldg(pm.bH[0] + i) * p + __ldg(pm.cH[0] + i) * dEy;
        tx += p;
    }
    if (sy >= 0) {
        R &p = s.phzy[(long long)sy * g.px + i];
        p = __ldg(pm.bH[1] + j) * p + __ldg(pm.cH[1] + j) * dEx;
        ty += p;
    }
    s.Hz[q] -= c.S * (tx - ty);
}

template <typename R>
__global__ void __launch_bounds__(BX *BY) k_hp(GeoP g, StateP<R> s, int slot, PmlP<R> pm)
{
    wait_previous_grid();
    h_cell<R>(g, s, coef_at<R>(slot), pm, blockIdx.x * BX + threadIdx.x, blockIdx.y * BY + threadIdx.y);
}

// Eq. (10a,b) for one edge of component cc at array index (i, j) with the
// scaled curl, the design / gap / source logic, records and sensitivity.
template <typename R, int MODE>
__device__ __forceinline__ void e_edge(const GeoP &g, const Coef<R> &c, const StepP<R> &a, int cc, int i, int j,
                                       R curl, R &E, R *J)
{
    const bool gap = in_range(i, g.g0[cc][0], g.gn[cc][0]) && in_range(j, g.g0[cc][1], g.gn[cc][1]);
    const int gidx = (cc ? g.Mgc[0] : 0) + (j - g.g0[cc][1]) * g.gn[cc][0] + (i - g.g0[cc][0]);
    const bool des = in_range(i, g.d0[cc][0], g.dn[cc][0]) && in_range(j, g.d0[cc][1], g.dn[cc][1]);
    const long long d = (long long)(j - g.d0[cc][1]) * g.dp[cc] + (i - g.dxa[cc]);
    R src = R(0);
    if (MODE == 0) {
        if (cc == 0 && in_range(i, g.s0[0], g.s1[0] - g.s0[0]) && in_range(j, g.s0[1], g.s1[1] - g.s0[1]))
            src = *a.src;
    } else if (gap) {
        src = -c.eps_g * a.gap_src[gidx];
    }
    const R e = E;
    R en;
    if (des && !gap) {
        const R rt = a.rho_t[cc][d];
        const R eps = c.eps_s + rt * c.d_eps;
        const R psi = c.psi_s + rt * (c.psi - c.psi_s);
        const R sig = c.sig_max * rt * (R(1) - rt);
        const R bJ = R(0.5) * psi * c.inv1g;
        const R hs = R(0.5) * (sig + bJ);
        const R cb = rcp(eps + hs);
        const R ca = (eps - hs) * cb;
        const R jo = J[d];
        en = ca * e + cb * (curl - c.half1pkJ * jo - src);
        const R jn = c.kJ * jo + bJ * (en + e);
        J[d] = jn;
        if (MODE == 0) {
            if (a.rec[cc]) a.rec[cc][d] = en;
        } else {
            // Eq. (25a-c) folded through the chain rule of Eq. (27).
            const R term = -c.t_eps * (en - e) - c.t_sig * (R(1) - R(2) * rt) * R(0.5) * (en + e) -
                           c.t_dpsi * rcp(psi) * R(0.5) * (jn + jo);
            a.G[cc][d] += (double)a.rec[cc][d] * (double)term;
        }
    } else {
        en = e + (curl - src) * (gap ? c.inv_eps_g : c.inv_eps_s);
        if (MODE == 0 && des && a.rec[cc]) a.rec[cc][d] = en;
    }
    E = en;
    if (MODE == 0 && gap && a.gap_rec) a.gap_rec[gidx] = en;
}

// E half step of the edges Ex(i, j) and Ey(i, j).
template <typename R, int MODE>
__device__ __forceinline__ void e_edges(const GeoP &g, const StateP<R> &s, const Coef<R> &c, const PmlP<R> &pm,
                                        const StepP<R> &a, int i, int j)
{
    if (i >= g.nx || j >= g.ny) return;
    const long long q = (long long)j * g.px + i;
    const int np = g.npml;
    // Ex(i, j): an edge of the grid (i <= nx-2) off the rows j = 0, ny-1
    const bool ux = i <= g.nx - 2 && j >= 1 && j <= g.ny - 2;
    // Ey(i, j): j <= ny-2, off the columns i = 0, nx-1
    const bool uy = j <= g.ny - 2 && i >= 1 && i <= g.nx - 2;
    R hz = R(0), hzS = R(0), hzW = R(0);
    if (ux || uy) hz = s.Hz[q];
    if (ux) hzS = s.Hz[q - g.px];
    if (uy) hzW = s.Hz[q - 1];
    if (ux) {
        const R d = hz - hzS;  // d_y Hz at (i+1/2, j)
        R t = d * __ldg(pm.kiE[1] + j);
        const int sy = slabE(j, g.ny, np);
        if (sy >= 0) {
            R &p = s.pexy[(long long)sy * g.px + i];
            p = __ldg(pm.bE[1] + j) * p + __ldg(pm.cE[1] + j) * d;
            t += p;
        }
        R ex = s.Ex[q];
        e_edge<R, MODE>(g, c, a, 0, i, j, c.S * t, ex, s.J[0]);
        s.Ex[q] = ex;
    }
    if (uy) {
        const R d = hz - hzW;  // d_x Hz at (i, j+1/2)
        R t = d * __ldg(pm.kiE[0] + i);
        const int sx = slabE(i, g.nx, np);
        if (sx >= 0) {
            R &p = s.peyx[(long long)j * 2 * np + sx];
            p = __ldg(pm.bE[0] + i) * p + __ldg(pm.cE[0] + i) * d;
            t += p;
        }
        R ey = s.Ey[q];
        e_edge<R, MODE>(g, c, a, 1, i, j, -c.S * t, ey, s.J[1]);
        s.Ey[q] = ey;
    }
}

template <typename R, int MODE>
__global__ void __launch_bounds__(BX *BY) k_ep(GeoP g, StateP<R> s, int slot, PmlP<R> pm, StepP<R> a)
{
    wait_previous_grid();
    e_edges<R, MODE>(g, s, coef_at<R>(slot), pm, a, blockIdx.x * BX + threadIdx.x, blockIdx.y * BY + threadIdx.y);
}

// ------------------------------------------------ several steps per launch
//
// On a small grid (the paper's 491^2 geometry holds 10 MB, resident in L2)
// each half step is a single partial wave, and the two launches of a step
// cost about their launch latency.  k_stepp_multi advances `count` steps in
// one cooperative launch (every block resident: one block of 1024 threads
// per SM), each half step a grid-stride sweep of the nodes followed by a
// grid-wide barrier: an arrival counter and a generation word in global
// memory, the last block to arrive releasing the others.  Waits are acquire
// loads bounded by `limit` clock cycles; on expiry the block records
// ERR_TIMEOUT and raises an abort word that every waiting block watches, so
// the whole grid returns.  Measured on the 491^2 geometry the barrier costs
// more than the launch boundary it replaces (12.4 against 6.1 us per step;
// a variant in which each 32 x 32 tile waits only for its four neighbours
// took 16.7 us), so contexts default to one launch per half step.

__device__ __forceinline__ unsigned load_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void store_release(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Wait (bounded) until *flag has reached `want` (counts modulo 2^32).
__device__ bool wait_flag(const unsigned *flag, unsigned want, unsigned *abort_word, unsigned *err, long long limit)
{
    const long long t0 = clock64();
    for (;;) {
        if ((int)(load_acquire(flag) - want) >= 0) return true;
        if (load_acquire(abort_word)) return false;
        if (clock64() - t0 > limit) {
            atomicOr(err, ERR_TIMEOUT);
            atomicExch(abort_word, 1u);
            return false;
        }
        __nanosleep(64);
    }
}

constexpr int GB = 1024;  // threads per block, one block per SM

// Grid-wide barrier: bar[0] counts arrivals, bar[1] is the generation the
// last arrival advances (bounded wait for it; false on expiry or abort).
__device__ __forceinline__ bool grid_sync(unsigned *bar, unsigned nblocks, unsigned *abort_word, unsigned *err,
                                          long long limit)
{
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned gen = load_acquire(bar + 1);
        __threadfence();
        bool ok = true;
        if (atomicAdd(bar, 1u) + 1 == nblocks) {
            bar[0] = 0;
            __threadfence();
            store_release(bar + 1, gen + 1);
        } else {
            ok = wait_flag(bar + 1, gen + 1, abort_word, err, limit);
        }
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

template <typename R, int MODE>
__global__ void __launch_bounds__(GB, 1) k_stepp_multi(GeoP g, StateP<R> s, int slot, PmlP<R> pm, StepP<R> base,
                                                       PlanP<R> plan, unsigned phase0, unsigned *flags,
                                                       unsigned *abort_word, unsigned *err, long long limit)
{
    const Coef<R> &c = coef_at<R>(slot);
    const int nx = g.nx, nn = g.nx * g.ny, stride = gridDim.x * GB;
    for (int t = 0; t < plan.count; ++t) {
        for (int q = blockIdx.x * GB + threadIdx.x; q < nn; q += stride) h_cell<R>(g, s, c, pm, q % nx, q / nx);
        if (!grid_sync(flags, gridDim.x, abort_word, err, limit)) return;
        StepP<R> a = base;
        if (MODE == 0) {
            const int n = plan.n0 + t;
            a.src = plan.src + n;
            a.gap_rec = plan.gap ? plan.gap + (long long)(n + 1) * plan.Mg : nullptr;
            R *sl = plan.rec ? plan.rec + (long long)(n - plan.rec0) * plan.rec_step : nullptr;
            a.rec[0] = sl;
            a.rec[1] = sl ? sl + plan.Mdi0 : nullptr;
        } else {
            const int m = plan.n0 - t;
            a.gap_src = plan.gap ? plan.gap + (long long)m * plan.Mg : nullptr;
            R *sl = plan.rec + (long long)(m - 1 - plan.rec0) * plan.rec_step;
            a.rec[0] = sl;
            a.rec[1] = sl + plan.Mdi0;
        }
        for (int q = blockIdx.x * GB + threadIdx.x; q < nn; q += stride) e_edges<R, MODE>(g, s, c, pm, a, q % nx, q / nx);
        if (!grid_sync(flags, gridDim.x, abort_word, err, limit)) return;
    }
}

// A wait on a flag nothing sets, for the self-test of the bounded wait.
__global__ void k_wait_selftest(unsigned *words, long long limit)
{
    if (threadIdx.x == 0) wait_flag(words, 1u, words + 1, words + 2, limit);
}

}  // namespace

template <typename R>
int launch_stepp(int mode, const GeoP &g, const StateP<R> &s, int c, const PmlP<R> &pm,
                 const StepP<R> &a, cudaStream_t st)
{
    const dim3 block(BX, BY), grid((g.nx + BX - 1) / BX, (g.ny + BY - 1) / BY);
    launch_pdl(k_hp<R>, grid, block, st, g, s, c, pm);
    if (mode == 0) launch_pdl(k_ep<R, 0>, grid, block, st, g, s, c, pm, a);
    else launch_pdl(k_ep<R, 1>, grid, block, st, g, s, c, pm, a);
    return 2;
}

int stepp_multi_tiles(const GeoP &) { return 2; }  // the barrier's arrival count and generation

template <typename R>
bool stepp_multi_fits(const GeoP &g)
{
    int dev = 0, sms = 0, per = 0, coop = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) {
        cudaGetLastError();
        return false;
    }
    int per1 = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_stepp_multi<R, 0>, GB, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per1, k_stepp_multi<R, 1>, GB, 0) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    per = per < per1 ? per : per1;
    return per >= 1;
}

template <typename R>
int launch_stepp_multi(int mode, const GeoP &g, const StateP<R> &s, int c, const PmlP<R> &pm, const StepP<R> &base,
                       const PlanP<R> &plan, unsigned phase0, unsigned *flags, unsigned *abort_word, unsigned *err,
                       long long limit, cudaStream_t st)
{
    cudaLaunchConfig_t cfg = {};
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cfg.gridDim = dim3((unsigned)sms);
    cfg.blockDim = dim3(GB);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (mode == 0)
        cudaLaunchKernelEx(&cfg, k_stepp_multi<R, 0>, g, s, c, pm, base, plan, phase0, flags, abort_word, err, limit);
    else
        cudaLaunchKernelEx(&cfg, k_stepp_multi<R, 1>, g, s, c, pm, base, plan, phase0, flags, abort_word, err, limit);
    return 1;
}

void launch_wait_selftest(unsigned *words, long long limit, cudaStream_t st)
{
    k_wait_selftest<<<1, 32, 0, st>>>(words, limit);
}

template bool stepp_multi_fits<float>(const GeoP &);
template bool stepp_multi_fits<double>(const GeoP &);
template int launch_stepp_multi<float>(int, const GeoP &, const StateP<float> &, int, const PmlP<float> &,
                                       const StepP<float> &, const PlanP<float> &, unsigned, unsigned *, unsigned *,
                                       unsigned *, long long, cudaStream_t);
template int launch_stepp_multi<double>(int, const GeoP &, const StateP<double> &, int, const PmlP<double> &,
                                        const StepP<double> &, const PlanP<double> &, unsigned, unsigned *,
                                        unsigned *, unsigned *, long long, cudaStream_t);
template int launch_stepp<float>(int, const GeoP &, const StateP<float> &, int, const PmlP<float> &,
                                 const StepP<float> &, cudaStream_t);
template int launch_stepp<double>(int, const GeoP &, const StateP<double> &, int,
                                  const PmlP<double> &, const StepP<double> &, cudaStream_t);

}  // namespace fdtd

namespace fdtd {
template <typename R>
cudaError_t upload_coef_p(int slot, const Coef<R> &c, cudaStream_t st)
{
    return write_coef_slot(slot, c, st);
}
template cudaError_t upload_coef_p<float>(int, const Coef<float> &, cudaStream_t);
template cudaError_t upload_coef_p<double>(int, const Coef<double> &, cudaStream_t);
}  // namespace fdtd
