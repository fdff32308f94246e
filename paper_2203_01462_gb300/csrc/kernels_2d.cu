// Fused 2D TM_z leapfrog step (Ez, Hx, Hy, Jz + CPML) for sm_103a.
//
// One launch advances the whole grid by one time step n -> n+1: the H half
// step of mu0 dH/dt = -curl E and the E half step of Eq. (10a,b) (J and
// sigma E averaged over the step, scaled units, see Coef).  State is read
// from one buffer of a ping-pong pair and written to the other, so every
// word crosses HBM once per step (24 B per vacuum node).
//
// Work layout: each thread owns one grid column and marches up a chunk of
// rows.  Values along y stay in registers (Ez of the next row, the new Hx of
// the previous row); x neighbours come from the adjacent lanes by warp
// shuffles.  A warp covers 32 columns but writes 31: lane 0 is a halo lane
// that recomputes the new Hy of the column left of the warp's first output
// column, and lane 31 loads Ez of the column to its right.  All region
// logic (CPML slabs, design box, gap, source row) is per column (fixed for
// the thread) or per row (uniform across the warp).
#include "fdtd_internal.h"

namespace fdtd {

namespace {

constexpr int WARPS = 4;
constexpr int NTH = 32 * WARPS;
constexpr int OUT_PER_WARP = 31;
constexpr int U = 4;  // rows loaded ahead per group

__device__ __forceinline__ bool in_range(int v, int lo, int n) { return (unsigned)(v - lo) < (unsigned)n; }

template <typename R, int MODE>
__global__ void __launch_bounds__(NTH, 6) k_step2d(Geo2D g, State2D<R> in, State2D<R> out, Coef<R> c, Pml1D<R> px,
                                                 Pml1D<R> py, TB2D<R> a, int chunk)
{
    const int lane = threadIdx.x & 31;
    const int warp = blockIdx.x * WARPS + (threadIdx.x >> 5);
    const int i = warp * OUT_PER_WARP - 1 + lane;  // this thread's column
    const int y0 = blockIdx.y * chunk;
    const int y1 = min(y0 + chunk, g.ny);
    const int nx = g.nx, ny = g.ny, np = g.npml;
    const size_t P = (size_t)g.px;

    const bool col = (unsigned)i < (unsigned)nx;
    const bool store = col && lane > 0;
    const bool colE = i >= 1 && i <= nx - 2;
    const bool hy_upd = col && i + 1 < nx;
    const bool xpE = col && np > 0 && (i < np || i >= nx - np);
    const bool xpH = col && np > 0 && (i < np || (i >= nx - 1 - np && i < nx - 1));
    const int slE = i < np ? i : i - (nx - 2 * np);
    const int slH = i < np ? i : np + i - (nx - 1 - np);
    const bool desx = in_range(i, g.dx0, g.dnx);
    const bool gapx = in_range(i, g.gx0, g.gnx);
    const bool srcx = in_range(i, g.sx0, g.sx1 - g.sx0);
    R kiEx = R(1), bEx = R(0), cEx = R(0), kiHx = R(1), bHx = R(0), cHx = R(0);
    if (xpE) { kiEx = px.kiE[i]; bEx = px.bE[i]; cEx = px.cE[i]; }
    if (xpH) { kiHx = px.kiH[i]; bHx = px.bH[i]; cHx = px.cH[i]; }
    const int n = a.n0;  // forward: step n; adjoint: m
    R src_val = R(0);
    if (MODE == 0 && srcx) src_val = a.src_tab[n];

    const R *__restrict__ iEz = in.Ez;
    const R *__restrict__ iHx = in.Hx;
    const R *__restrict__ iHy = in.Hy;
    auto ld = [&](const R *__restrict__ p, int j) -> R {
        return (col && (unsigned)j < (unsigned)ny) ? p[(size_t)j * P + i] : R(0);
    };

    // New Hx of row j from old Hx, Ez(j), Ez(j+1) and (in a y-slab) the old
    // CPML term psi_old; the new term goes to *psi_new.
    auto hx_new = [&](int j, R hx, R ez, R ezn, R psi_old, R *psi_new) -> R {
        if (j + 1 >= ny || !col) return hx;
        const R d = ezn - ez;
        R t = d;
        if (np > 0 && (j < np || j >= ny - 1 - np)) {
            const R p = py.bH[j] * psi_old + py.cH[j] * d;
            *psi_new = p;
            t = d * py.kiH[j] + p;
        }
        return hx - c.S * t;
    };
    auto yslabH = [&](int j) { return np > 0 && j + 1 < ny && (j < np || j >= ny - 1 - np); };
    auto yslabE = [&](int j) { return np > 0 && (j < np || j >= ny - np); };
    auto slabH = [&](int j) { return j < np ? j : np + j - (ny - 1 - np); };
    auto slabE = [&](int j) { return j < np ? j : j - (ny - 2 * np); };

    // Prologue: Ez of the first row and the new Hx of the row below it.
    R ez = ld(iEz, y0);
    R hxp = R(0);
    if (y0 >= 1) {
        R dummy;
        const R po = (col && yslabH(y0 - 1)) ? in.phxy[(size_t)slabH(y0 - 1) * P + i] : R(0);
        hxp = hx_new(y0 - 1, ld(iHx, y0 - 1), ld(iEz, y0 - 1), ez, po, &dummy);
    }

    // Warp-uniform classification of the warp's columns: a row group takes
    // the fast path when no column of the warp and no row of the group
    // touches a wall, a CPML slab, the design box, the gap or the source.
    const unsigned FULL = 0xffffffffu;
    // Lane 0 only supplies the new Hy of its column, so it needs a plain H
    // update there; the other lanes need a plain E update too.
    const bool plain_col = col && (lane == 0 ? (hy_upd && !xpH) : (colE && !xpE && !xpH));
    const bool wx_edge = !__all_sync(FULL, plain_col);
    const bool wx_des = __any_sync(FULL, desx && lane > 0);
    const bool wx_src = __any_sync(FULL, srcx && lane > 0);

    for (int jb = y0; jb < y1; jb += U) {
        const int je = min(jb + U, y1);
        const bool rows_ok = jb >= 1 && je + 1 <= ny - 1 && !(np > 0 && (jb < np + 1 || je > ny - 2 - np));
        const bool rows_des = in_range(jb, g.dy0 - U + 1, g.dny + U - 1);
        const bool rows_src = jb < g.sy1 && je > g.sy0;
        const bool fast = !wx_edge && rows_ok && !(wx_des && rows_des) && !(wx_src && rows_src) && je - jb == U;
        if (fast) {
            R ezn_[U], hx_[U], hy_[U], ezr_[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const size_t q = (size_t)(jb + u) * P + i;
                ezn_[u] = iEz[q + P];
                hx_[u] = iHx[q];
                hy_[u] = iHy[q];
                ezr_[u] = lane == 31 ? iEz[q + 1] : R(0);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const size_t q = (size_t)(jb + u) * P + i;
                R ezr = __shfl_down_sync(FULL, ez, 1);
                if (lane == 31) ezr = ezr_[u];
                const R hxn = hx_[u] - c.S * (ezn_[u] - ez);
                const R hyn = hy_[u] + c.S * (ezr - ez);
                const R hyl = __shfl_up_sync(FULL, hyn, 1);
                const R en = ez + c.S * c.inv_eps_s * ((hyn - hyl) - (hxn - hxp));
                if (lane > 0) {
                    out.Ez[q] = en;
                    out.Hx[q] = hxn;
                    out.Hy[q] = hyn;
                }
                ez = ezn_[u];
                hxp = hxn;
            }
            continue;
        }

        // ---- general path: loads of the group first, CPML terms on demand
        R ezn_[U], hx_[U], hy_[U], ezr_[U], J_[U], rt_[U], em_[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = jb + u;
            ezn_[u] = ld(iEz, j + 1);
            hx_[u] = ld(iHx, j);
            hy_[u] = ld(iHy, j);
            ezr_[u] = (lane == 31 && col && i + 1 < nx && j < ny) ? iEz[(size_t)j * P + i + 1] : R(0);
            const bool des = desx && in_range(j, g.dy0, g.dny) && j < y1;
            const size_t d = (size_t)(j - g.dy0) * g.dnx + (i - g.dx0);
            J_[u] = des ? in.J[d] : R(0);
            rt_[u] = des ? a.rho_t[d] : R(0);
            em_[u] = (MODE == 1 && des) ? a.rec[(size_t)(n - 1 - a.slot0) * a.Md + d] : R(0);
        }

#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = jb + u;
            if (j >= y1) break;
            const size_t q = (size_t)j * P + i;
            const R ezn = ezn_[u];
            R ezr = __shfl_down_sync(FULL, ez, 1);
            if (lane == 31) ezr = ezr_[u];

            // ---- H half step
            R psn = R(0);
            const R pho = (col && yslabH(j)) ? in.phxy[(size_t)slabH(j) * P + i] : R(0);
            const R hxn = hx_new(j, hx_[u], ez, ezn, pho, &psn);
            if (store && yslabH(j)) out.phxy[(size_t)slabH(j) * P + i] = psn;
            R hyn = hy_[u];
            if (hy_upd) {
                const R dd = ezr - ez;
                R t = dd;
                if (xpH) {
                    const size_t qs = (size_t)j * 2 * np + slH;
                    const R p = bHx * in.phyx[qs] + cHx * dd;
                    if (store) out.phyx[qs] = p;
                    t = dd * kiHx + p;
                }
                hyn = hy_[u] + c.S * t;
            }
            const R hyl = __shfl_up_sync(FULL, hyn, 1);

            // ---- E (and J) half step
            R en = ez;
            const bool rowE = j >= 1 && j <= ny - 2;
            if (colE && rowE) {
                const R dHy = hyn - hyl;
                const R dHx = hxn - hxp;
                R cx = dHy, cy = dHx;
                if (xpE) {
                    const size_t qs = (size_t)j * 2 * np + slE;
                    const R p = bEx * in.pezx[qs] + cEx * dHy;
                    if (store) out.pezx[qs] = p;
                    cx = dHy * kiEx + p;
                }
                if (yslabE(j)) {
                    const size_t qs = (size_t)slabE(j) * P + i;
                    const R p = py.bE[j] * in.pezy[qs] + py.cE[j] * dHx;
                    if (store) out.pezy[qs] = p;
                    cy = dHx * py.kiE[j] + p;
                }
                const R curl = c.S * (cx - cy);
                const bool gap = gapx && in_range(j, g.gy0, g.gny);
                const int gidx = (j - g.gy0) * g.gnx + (i - g.gx0);
                R src = R(0);
                if (MODE == 0) {
                    if (srcx && in_range(j, g.sy0, g.sy1 - g.sy0)) src = src_val;
                } else if (gap) {
                    src = -c.eps_g * a.gap_hist[(size_t)n * a.Mg + gidx];
                }
                const bool des = desx && in_range(j, g.dy0, g.dny);
                const size_t d = (size_t)(j - g.dy0) * g.dnx + (i - g.dx0);
                if (des && !gap) {
                    const R rt = rt_[u];
                    const R eps = c.eps_s + rt * c.d_eps;
                    const R psi = c.psi_s + rt * (c.psi - c.psi_s);
                    const R sig = c.sig_max * rt * (R(1) - rt);
                    const R bJ = R(0.5) * psi * c.inv1g;
                    const R hs = R(0.5) * (sig + bJ);
                    const R cb = R(1) / (eps + hs);
                    const R ca = (eps - hs) * cb;
                    const R jo = J_[u];
                    en = ca * ez + cb * (curl - c.half1pkJ * jo - src);
                    const R jn = c.kJ * jo + bJ * (en + ez);
                    if (store) {
                        out.J[d] = jn;
                        if (MODE == 0) {
                            if (a.rec) a.rec[d] = en;
                        } else {
                            // Eq. (25a-c) folded through the chain rule of Eq. (27).
                            const R term = -c.d_eps * (en - ez) -
                                           c.sig_max * (R(1) - R(2) * rt) * R(0.5) * (en + ez) -
                                           ((c.psi - c.psi_s) / psi) * R(0.5) * (jn + jo);
                            a.G[d] += (double)em_[u] * (double)term;
                        }
                    }
                } else {
                    en = ez + (curl - src) * (gap ? c.inv_eps_g : c.inv_eps_s);
                    if (MODE == 0 && store && des && a.rec) a.rec[d] = en;
                }
                if (MODE == 0 && store && gap && a.gap_rec) a.gap_rec[(size_t)(n + 1) * a.Mg + gidx] = en;
            }
            if (store) {
                out.Ez[q] = en;
                out.Hx[q] = hxn;
                out.Hy[q] = hyn;
            }
            ez = ezn;
            hxp = hxn;
        }
    }
}

}  // namespace

template <typename R>
int launch_step2d(int mode, int chunk, const Geo2D &g, const State2D<R> &in, const State2D<R> &out, const Coef<R> &c,
                  const Pml1D<R> &px, const Pml1D<R> &py, const TB2D<R> &a, cudaStream_t st)
{
    const int warps = (g.nx + 1 + OUT_PER_WARP - 1) / OUT_PER_WARP;
    dim3 grid((warps + WARPS - 1) / WARPS, (g.ny + chunk - 1) / chunk);
    if (mode == 0) k_step2d<R, 0><<<grid, NTH, 0, st>>>(g, in, out, c, px, py, a, chunk);
    else k_step2d<R, 1><<<grid, NTH, 0, st>>>(g, in, out, c, px, py, a, chunk);
    return 1;
}

template int launch_step2d<float>(int, int, const Geo2D &, const State2D<float> &, const State2D<float> &,
                                  const Coef<float> &, const Pml1D<float> &, const Pml1D<float> &,
                                  const TB2D<float> &, cudaStream_t);
template int launch_step2d<double>(int, int, const Geo2D &, const State2D<double> &, const State2D<double> &,
                                   const Coef<double> &, const Pml1D<double> &, const Pml1D<double> &,
                                   const TB2D<double> &, cudaStream_t);

}  // namespace fdtd
