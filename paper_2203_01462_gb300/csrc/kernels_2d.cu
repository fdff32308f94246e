// 2D TM_z stencil kernels (Ez, Hx, Hy, Jz) for sm_103a.
//
// Sec. 3.2 of the paper: Yee grid, E and the Drude current J at integer time
// steps, H at half steps.  The H half-step is mu0 dH/dt = -curl E; the E half
// step solves Eq. (10a,b) per node with J and sigma E averaged over the step
// (the ADE reading used throughout), in scaled units (see Coef).  CPML terms
// are updated only in the border slabs.
//
// One thread per node; the kernels are bandwidth-bound, so the design aims
// at coalesced row access (x fastest, 32-wide warps along x).
#include "fdtd_internal.h"

namespace fdtd {

namespace {

constexpr int BX = 32, BY = 8;

__device__ __forceinline__ bool in_range(int v, int lo, int n) { return (unsigned)(v - lo) < (unsigned)n; }

// H^{n-1/2} -> H^{n+1/2} from E^n.  Hx[j][i] needs Ez(i, j+1), Hy[j][i]
// needs Ez(i+1, j); the last row / column of Hx / Hy is outside the grid.
template <typename R>
__global__ void __launch_bounds__(BX *BY) k_h2d(Geo2D g, State2D<R> s, Coef<R> c, Pml1D<R> px, Pml1D<R> py)
{
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    const size_t q = (size_t)j * g.px + i;
    const R e = s.Ez[q];
    const int np = g.npml;
    if (j + 1 < g.ny) {
        const R d = s.Ez[q + g.px] - e;
        R t = d * py.kiH[j];
        int sl = -1;
        if (j < np) sl = j;
        else if (j >= g.ny - 1 - np) sl = np + j - (g.ny - 1 - np);
        if (sl >= 0) {
            R &p = s.phxy[(size_t)sl * g.px + i];
            p = py.bH[j] * p + py.cH[j] * d;
            t += p;
        }
        s.Hx[q] -= c.S * t;
    }
    if (i + 1 < g.nx) {
        const R d = s.Ez[q + 1] - e;
        R t = d * px.kiH[i];
        int sl = -1;
        if (i < np) sl = i;
        else if (i >= g.nx - 1 - np) sl = np + i - (g.nx - 1 - np);
        if (sl >= 0) {
            R &p = s.phyx[(size_t)j * 2 * np + sl];
            p = px.bH[i] * p + px.cH[i] * d;
            t += p;
        }
        s.Hy[q] += c.S * t;
    }
}

// (E, J)^n -> (E, J)^{n+1} from H^{n+1/2}.  PEC walls: the outermost Ez
// nodes are never written.  MODE 0: forward (source from the table, gap and
// design-box records); MODE 1: adjoint (source eps_g E^m in the gap,
// sensitivity accumulation of Eq. (25) in the design box).
template <typename R, int MODE>
__global__ void __launch_bounds__(BX *BY) k_e2d(Geo2D g, State2D<R> s, Coef<R> c, Pml1D<R> px, Pml1D<R> py,
                                               Step2D<R> a)
{
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    if (i < 1 || j < 1 || i >= g.nx - 1 || j >= g.ny - 1) return;
    const size_t q = (size_t)j * g.px + i;
    const int np = g.npml;
    const R dHy = s.Hy[q] - s.Hy[q - 1];
    const R dHx = s.Hx[q] - s.Hx[q - g.px];
    R cx = dHy * px.kiE[i];
    R cy = dHx * py.kiE[j];
    {
        int sl = -1;
        if (i < np) sl = i;
        else if (i >= g.nx - np) sl = i - (g.nx - 2 * np);
        if (sl >= 0) {
            R &p = s.pezx[(size_t)j * 2 * np + sl];
            p = px.bE[i] * p + px.cE[i] * dHy;
            cx += p;
        }
    }
    {
        int sl = -1;
        if (j < np) sl = j;
        else if (j >= g.ny - np) sl = j - (g.ny - 2 * np);
        if (sl >= 0) {
            R &p = s.pezy[(size_t)sl * g.px + i];
            p = py.bE[j] * p + py.cE[j] * dHx;
            cy += p;
        }
    }
    const R curl = c.S * (cx - cy);

    const bool gap = in_range(i, g.gx0, g.gnx) && in_range(j, g.gy0, g.gny);
    const int gidx = (j - g.gy0) * g.gnx + (i - g.gx0);
    R src = R(0);
    if (MODE == 0) {
        if (in_range(i, g.sx0, g.sx1 - g.sx0) && in_range(j, g.sy0, g.sy1 - g.sy0)) src = *a.src;
    } else if (gap) {
        src = -c.eps_g * a.gap_src[gidx];
    }

    const R e = s.Ez[q];
    const bool des = in_range(i, g.dx0, g.dnx) && in_range(j, g.dy0, g.dny);
    const size_t d = (size_t)(j - g.dy0) * g.dnx + (i - g.dx0);
    R en;
    if (des && !gap) {
        const R rt = a.rho_t[d];
        const R eps = c.eps_s + rt * c.d_eps;
        const R psi = c.psi_s + rt * (c.psi - c.psi_s);
        const R sig = c.sig_max * rt * (R(1) - rt);
        const R bJ = R(0.5) * psi * c.inv1g;
        const R hs = R(0.5) * (sig + bJ);
        const R cb = R(1) / (eps + hs);
        const R ca = (eps - hs) * cb;
        const R jo = s.J[d];
        en = ca * e + cb * (curl - c.half1pkJ * jo - src);
        const R jn = c.kJ * jo + bJ * (en + e);
        s.J[d] = jn;
        if (MODE == 0) {
            if (a.rec) a.rec[d] = en;
        } else {
            // Eq. (25) folded through the chain rule of Eq. (27):
            // -d_eps (E*' - E*) - sig_max (1 - 2 rho~) (E*' + E*) / 2
            // - ((psi - psi_s) / psi_i) (J*' + J*) / 2, times forward E^m.
            const R term = -c.d_eps * (en - e) - c.sig_max * (R(1) - R(2) * rt) * R(0.5) * (en + e) -
                           ((c.psi - c.psi_s) / psi) * R(0.5) * (jn + jo);
            a.G[d] += (double)a.rec[d] * (double)term;
        }
    } else {
        en = e + (curl - src) * (gap ? c.inv_eps_g : c.inv_eps_s);
        if (MODE == 0 && des && a.rec) a.rec[d] = en;
    }
    s.Ez[q] = en;
    if (MODE == 0 && gap && a.gap_rec) a.gap_rec[gidx] = en;
}

}  // namespace

template <typename R>
void launch_h2d(const Geo2D &g, const State2D<R> &s, const Coef<R> &c, const Pml1D<R> &px,
                const Pml1D<R> &py, cudaStream_t st)
{
    dim3 b(BX, BY), gr((g.nx + BX - 1) / BX, (g.ny + BY - 1) / BY);
    k_h2d<R><<<gr, b, 0, st>>>(g, s, c, px, py);
}

template <typename R>
void launch_e2d(int mode, const Geo2D &g, const State2D<R> &s, const Coef<R> &c, const Pml1D<R> &px,
                const Pml1D<R> &py, const Step2D<R> &a, cudaStream_t st)
{
    dim3 b(BX, BY), gr((g.nx + BX - 1) / BX, (g.ny + BY - 1) / BY);
    if (mode == 0) k_e2d<R, 0><<<gr, b, 0, st>>>(g, s, c, px, py, a);
    else k_e2d<R, 1><<<gr, b, 0, st>>>(g, s, c, px, py, a);
}

template void launch_h2d<float>(const Geo2D &, const State2D<float> &, const Coef<float> &,
                                const Pml1D<float> &, const Pml1D<float> &, cudaStream_t);
template void launch_h2d<double>(const Geo2D &, const State2D<double> &, const Coef<double> &,
                                 const Pml1D<double> &, const Pml1D<double> &, cudaStream_t);
template void launch_e2d<float>(int, const Geo2D &, const State2D<float> &, const Coef<float> &,
                                const Pml1D<float> &, const Pml1D<float> &, const Step2D<float> &,
                                cudaStream_t);
template void launch_e2d<double>(int, const Geo2D &, const State2D<double> &, const Coef<double> &,
                                 const Pml1D<double> &, const Pml1D<double> &, const Step2D<double> &,
                                 cudaStream_t);

}  // namespace fdtd
