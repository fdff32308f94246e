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

template <typename R>
__global__ void __launch_bounds__(BX *BY) k_hp(GeoP g, StateP<R> s, int slot, PmlP<R> pm)
{
    wait_previous_grid();
    const Coef<R> &c = coef_at<R>(slot);
    const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
    if (i > g.nx - 2 || j > g.ny - 2) return;  // Hz exists on the (nx-1) x (ny-1) cells
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

template <typename R, int MODE>
__global__ void __launch_bounds__(BX *BY) k_ep(GeoP g, StateP<R> s, int slot, PmlP<R> pm, StepP<R> a)
{
    wait_previous_grid();
    const Coef<R> &c = coef_at<R>(slot);
    const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
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
