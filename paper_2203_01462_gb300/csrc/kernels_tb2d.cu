// Temporally blocked 2D TM_z leapfrog (Ez, Hx, Hy, Jz + CPML) for small
// grids, for sm_103a.
//
// On a small grid (the surrogate workload's 316^2, the 160^2 parity case)
// each launch-per-step kernel is a single partial wave, so a step costs a
// few launch and memory latencies (about 7 us) whatever its work.  Here a
// block (one thread per column of the region, its rows in passes of 16)
// owns a square tile of 16 to 32 nodes a side (the smallest whose tiles
// fill at most one wave of blocks, one block per SM: 27 at 316^2, 14 x 14
// instead of 10 x 10 of 32 on 152 SMs, for 20 % less work per block); one
// launch advances T steps (T <= TB_MAX in
// FP32, 4 in FP64) at once.  The block loads its tile with a halo of T
// nodes on every side into shared memory (fields, J and the Drude
// coefficients of rho~ on design nodes, the CPML terms on slab nodes), runs
// the T steps there (an H half step and an E half step per step, each over
// the whole region, separated by block barriers), and writes back only its
// own tile, from one buffer of the ping-pong pair into the other.  Each half
// step invalidates one layer of the region from the outside (H reads Ez one
// node up and right, E reads H one node down and left), so after T steps
// the tile itself is still exact and no block ever waits for another.
// Records (the gap history, the design-box history), the source and, in the
// adjoint, the forward record and the FP64 sensitivity accumulator are read
// and written for the tile's own nodes only; the adjoint's records of all T
// steps are loaded with the tile, so no global load waits inside the step
// loop.
//
// Everything about a node that does not change from step to step is worked
// out once per launch: which half-step updates exist there (walls, region
// edge), whether it lies in a CPML slab, the design box, the gap, the
// source row or the block's own tile (one flag word per node, in
// registers), the Drude coefficients of its rho~, and the CPML tables of
// the region's rows and columns (staged in shared memory).  The region's
// arrays have a fixed row stride (the widest region), so every neighbour of
// a node is a constant offset from one address.  The step loop then does
// only the update arithmetic, which is that of the launch-per-step kernel's
// generic (border) path: H -= S t / H += S t with t the CPML-corrected
// difference, E from the curl S (c_x - c_y) through the same Drude, gap and
// source update.

#include <algorithm>

#include "coef_slots.cuh"
#include "fdtd_internal.h"

namespace fdtd {

namespace {

constexpr int TBT = 32;  // largest tile side (nodes); a launch's tile side w.tile is 16 .. 32
constexpr int TBY = 16;  // threads along y (region rows in passes of TBY)

// Region geometry per precision: most steps per launch, row stride (the
// widest region, TBT + 2 TM nodes), threads along x (one per column) and
// rows per thread.
template <typename R>
struct Dim {
    static constexpr int TM = sizeof(R) == 4 ? TB_MAX : 4;
    static constexpr int RW = TBT + 2 * TM;
    static constexpr int RC = RW * RW;
    static constexpr int NTH = RW * TBY;
    static constexpr int NK = (RW + TBY - 1) / TBY;
};

__device__ __forceinline__ bool in_range(int v, int lo, int n) { return (unsigned)(v - lo) < (unsigned)n; }
__device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp(double x) { return __drcp_rn(x); }

// Slab indices of the CPML arrays: x-slab columns [ny][2 np] and y-slab rows
// [2 np][px], for E (node positions) and H (half positions); -1 outside.
__device__ __forceinline__ int slab_e(int p, int n, int np) { return p < np ? p : (p >= n - np ? p - (n - 2 * np) : -1); }
__device__ __forceinline__ int slab_h(int p, int n, int np)
{
    return p < np ? p : ((p >= n - 1 - np && p < n - 1) ? np + p - (n - 1 - np) : -1);
}

// Per-node flags (fixed for a launch).
enum : unsigned {
    F_HX = 1u,       // Hx updated here (a row above exists in the grid and the region)
    F_HY = 2u,       // Hy updated here (a column to the right exists)
    F_HXP = 4u,      // ... with its y-slab CPML term
    F_HYP = 8u,      // ... with its x-slab CPML term
    F_E = 16u,       // Ez updated here (off the walls, not on the region's first row / column)
    F_EXP = 32u,     // ... with its x-slab CPML term
    F_EYP = 64u,     // ... with its y-slab CPML term
    F_DRU = 128u,    // Drude update: design box, not gap
    F_DES = 256u,    // design box (its E is recorded)
    F_GAP = 512u,    // gap
    F_SRC = 1024u,   // source row (forward)
    F_OWN = 2048u,   // the block's own tile
};

// Shared-memory arrays of one block: RARR region arrays [RC] (R), the CPML
// tables of the region's columns (x) and rows (y) [NTAB][RW] (R), the
// adjoint's records [T][TBT][TBT] (R) and its accumulator [TBT][TBT]
// (double).  On design nodes ca, cb, bJ (and, for the adjoint's
// sensitivity bracket, a1, a2) are the Drude update's coefficients, worked
// out from rho~ once per launch exactly as the step kernel's drude() works
// them out every step.
constexpr int RARR = 13;
constexpr int NTAB = 12;  // x: bE cE kE bH cH kH, then y: the same
template <typename R>
struct Region {
    R *ez, *hx, *hy, *J, *ca, *cb, *bJ, *a1, *a2, *pezx, *phyx, *pezy, *phxy;
    R *tab, *rec;
    double *G;
};

template <typename R>
__device__ __forceinline__ Region<R> carve_region(char *base, int T)
{
    constexpr int RC = Dim<R>::RC, RW = Dim<R>::RW;
    Region<R> r;
    R *p = (R *)base;
    r.ez = p;
    r.hx = p + RC;
    r.hy = p + 2 * RC;
    r.J = p + 3 * RC;
    r.ca = p + 4 * RC;
    r.cb = p + 5 * RC;
    r.bJ = p + 6 * RC;
    r.a1 = p + 7 * RC;
    r.a2 = p + 8 * RC;
    r.pezx = p + 9 * RC;
    r.phyx = p + 10 * RC;
    r.pezy = p + 11 * RC;
    r.phxy = p + 12 * RC;
    r.tab = p + RARR * RC;
    r.rec = r.tab + NTAB * RW;
    // the accumulator after the T record planes, 16-byte aligned
    size_t off = (size_t)(RARR * RC + NTAB * RW + T * TBT * TBT) * sizeof(R);
    off = (off + 15) & ~(size_t)15;
    r.G = (double *)(base + off);
    return r;
}

}  // namespace

// Shared memory of one block for steps of at most T per launch.
size_t tb2d_smem_bytes(int esz, int T)
{
    const int RW = TBT + 2 * (esz == 4 ? TB_MAX : 4);
    size_t off = (size_t)(RARR * RW * RW + NTAB * RW + T * TBT * TBT) * esz;
    off = (off + 15) & ~(size_t)15;
    return off + (size_t)TBT * TBT * sizeof(double);
}

// Tile side for an nx x ny grid: the smallest side in 16 .. 32 whose tiles
// fit in one wave of `sms` blocks (the block's region, and so its work per
// step, shrinks with the side), else 32.
int tb2d_tile(int nx, int ny, int sms)
{
    for (int t = 16; t < TBT; ++t)
        if ((long long)((nx + t - 1) / t) * ((ny + t - 1) / t) <= sms) return t;
    return TBT;
}

namespace {

template <typename R, int MODE>
__global__ void __launch_bounds__(Dim<R>::NTH, 1)
    k_tb2d(const __grid_constant__ Geo2D g, const __grid_constant__ State2D<R> in,
           const __grid_constant__ State2D<R> out, int slot, const __grid_constant__ Pml1D<R> px,
           const __grid_constant__ Pml1D<R> py, const __grid_constant__ Tb2D<R> w)
{
    constexpr int RW = Dim<R>::RW, NK = Dim<R>::NK, NTH = Dim<R>::NTH;
    extern __shared__ __align__(16) char smem[];
    const int T = w.count, tb = w.tile, side = tb + 2 * T;
    const Region<R> r = carve_region<R>(smem, T);
    const Coef<R> &c = coef_at<R>(slot);
    const int nx = g.nx, ny = g.ny, np = g.npml, P = g.px, np2 = 2 * np;
    const int x0 = blockIdx.x * tb - T, y0 = blockIdx.y * tb - T;  // region origin (global)
    const int tx = threadIdx.x, ty = threadIdx.y;
    const R S = c.S;
    const int Mg = g.gnx * g.gny;
    // the source amplitudes of the launch's steps, loaded with the tile
    __shared__ R src_s[TB_MAX];
    if (MODE == 0 && ty == 0 && tx < T) src_s[tx] = w.src[w.n0 + tx];

    // ---- CPML tables of the region's columns (x: ty 0) and rows (y: ty 1):
    // b, c, 1/kappa at node positions (E), then at half positions (H)
    if (ty < 2 && tx < side) {
        const int p = (ty == 0 ? x0 : y0) + tx, n = ty == 0 ? nx : ny;
        const Pml1D<R> &t = ty == 0 ? px : py;
        R v[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
        if (np > 0 && (unsigned)p < (unsigned)n) {
            v[0] = t.bE[p];
            v[1] = t.cE[p];
            v[2] = t.kiE[p];
            v[3] = t.bH[p];
            v[4] = t.cH[p];
            v[5] = t.kiH[p];
        }
#pragma unroll
        for (int a = 0; a < 6; ++a) r.tab[(ty * 6 + a) * RW + tx] = v[a];
    }

    // ---- load the region (zeros outside the grid and outside the boxes) and
    // work out each node's flags.  Each thread owns column ri = tx of the
    // region and its rows ty + k TBY, k < NK, here and in the step loop.
    const int ri = tx, i = x0 + ri;
    unsigned fk[NK];
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        const int rj = ty + k * TBY, j = y0 + rj, q = rj * RW + ri;
        unsigned f = 0;
        if (rj < RW) {
            R ez = R(0), hx = R(0), hy = R(0), J = R(0), a = R(0), b = R(0), cc = R(0), d = R(0);
            R ca = R(0), cb = R(0), bJ = R(0), a1 = R(0), a2 = R(0);
            if (ri < side && rj < side && (unsigned)i < (unsigned)nx && (unsigned)j < (unsigned)ny) {
                const long long gq = (long long)j * P + i;
                ez = in.Ez[gq];
                hx = in.Hx[gq];
                hy = in.Hy[gq];
                const bool des = in_range(i, g.dx0, g.dnx) && in_range(j, g.dy0, g.dny);
                const bool gap = in_range(i, g.gx0, g.gnx) && in_range(j, g.gy0, g.gny);
                if (des) {
                    const long long dg = (long long)(j - g.dy0) * g.dp + (i - g.dxa);
                    J = in.J[dg];
                    // the coefficients of drude(), in its order of operations
                    const R rt = w.rho_t[dg];
                    const R eps = c.eps_s + rt * c.d_eps;
                    const R psi = c.psi_s + rt * (c.psi - c.psi_s);
                    const R sig = c.sig_max * rt * (R(1) - rt);
                    bJ = R(0.5) * psi * c.inv1g;
                    const R hs = R(0.5) * (sig + bJ);
                    cb = rcp(eps + hs);
                    ca = (eps - hs) * cb;
                    if (MODE == 1) {
                        a1 = c.t_sig * (R(1) - R(2) * rt) * R(0.5);
                        a2 = c.t_dpsi * rcp(psi) * R(0.5);
                    }
                }
                if (np > 0) {
                    const int se = slab_e(i, nx, np), sh = slab_h(i, nx, np);
                    const int te = slab_e(j, ny, np), th = slab_h(j, ny, np);
                    if (se >= 0) a = in.pezx[(long long)j * np2 + se];
                    if (sh >= 0) b = in.phyx[(long long)j * np2 + sh];
                    if (te >= 0) cc = in.pezy[(long long)te * P + i];
                    if (th >= 0) d = in.phxy[(long long)th * P + i];
                }
                if (j + 1 < ny && rj + 1 < side) {
                    f |= F_HX;
                    if (np > 0 && (j < np || j >= ny - 1 - np)) f |= F_HXP;
                }
                if (i + 1 < nx && ri + 1 < side) {
                    f |= F_HY;
                    if (np > 0 && (i < np || i >= nx - 1 - np)) f |= F_HYP;
                }
                if (i >= 1 && i <= nx - 2 && j >= 1 && j <= ny - 2 && ri >= 1 && rj >= 1) {
                    f |= F_E;
                    if (np > 0 && (i < np || i >= nx - np)) f |= F_EXP;
                    if (np > 0 && (j < np || j >= ny - np)) f |= F_EYP;
                }
                if (des) f |= F_DES;
                if (des && !gap) f |= F_DRU;
                if (gap) f |= F_GAP;
                if (MODE == 0 && in_range(i, g.sx0, g.sx1 - g.sx0) && in_range(j, g.sy0, g.sy1 - g.sy0)) f |= F_SRC;
                if (ri >= T && ri < T + tb && rj >= T && rj < T + tb) f |= F_OWN;
            }
            r.ez[q] = ez;
            r.hx[q] = hx;
            r.hy[q] = hy;
            r.J[q] = J;
            r.ca[q] = ca;
            r.cb[q] = cb;
            r.bJ[q] = bJ;
            r.a1[q] = a1;
            r.a2[q] = a2;
            r.pezx[q] = a;
            r.phyx[q] = b;
            r.pezy[q] = cc;
            r.phxy[q] = d;
        }
        fk[k] = f;
    }
    // (adjoint) the accumulator of the tile's own nodes and their forward
    // records of all T steps
    const int flat = ty * RW + tx;
    if (MODE == 1)
        for (int o = flat; o < tb * tb; o += NTH) {
            const int oi = blockIdx.x * tb + o % tb, oj = blockIdx.y * tb + o / tb;
            const bool des = oi < nx && oj < ny && in_range(oi, g.dx0, g.dnx) && in_range(oj, g.dy0, g.dny);
            const long long dg = (long long)(oj - g.dy0) * g.dp + (oi - g.dxa);
            r.G[o] = des ? w.G[dg] : 0.0;
            for (int t = 0; t < T; ++t)
                r.rec[t * TBT * TBT + o] = des ? w.rec[(long long)(w.n0 - t - 1 - w.rec0) * w.Mdi + dg] : R(0);
        }
    __syncthreads();

    const int q0 = ty * RW + ri;
    for (int t = 0; t < T; ++t) {
        // ---- H half step over the region (reads Ez, writes Hx, Hy, psi_H);
        // every thread loads the inputs of all its rows before it computes
        // any of them (the loads of different rows then overlap)
        {
            R ez[NK], ezU[NK], ezR[NK], hxo[NK], hyo[NK], pxy[NK], pyx[NK];
#pragma unroll
            for (int k = 0; k < NK; ++k) {
                const unsigned f = fk[k];
                const int q = q0 + k * TBY * RW;
                ez[k] = ezU[k] = ezR[k] = hxo[k] = hyo[k] = pxy[k] = pyx[k] = R(0);
                if (f & (F_HX | F_HY)) ez[k] = r.ez[q];
                if (f & F_HX) {
                    ezU[k] = r.ez[q + RW];
                    hxo[k] = r.hx[q];
                }
                if (f & F_HY) {
                    ezR[k] = r.ez[q + 1];
                    hyo[k] = r.hy[q];
                }
                if (f & F_HXP) pxy[k] = r.phxy[q];
                if (f & F_HYP) pyx[k] = r.phyx[q];
            }
#pragma unroll
            for (int k = 0; k < NK; ++k) {
                const unsigned f = fk[k];
                const int q = q0 + k * TBY * RW, rj = ty + k * TBY;
                if (f & F_HX) {
                    const R dd = ezU[k] - ez[k];
                    R tt = dd;
                    if (f & F_HXP) {  // y tables at half positions: rows 9, 10, 11
                        const R p = r.tab[9 * RW + rj] * pxy[k] + r.tab[10 * RW + rj] * dd;
                        r.phxy[q] = p;
                        tt = dd * r.tab[11 * RW + rj] + p;
                    }
                    r.hx[q] = hxo[k] - S * tt;
                }
                if (f & F_HY) {
                    const R dd = ezR[k] - ez[k];
                    R tt = dd;
                    if (f & F_HYP) {  // x tables at half positions: rows 3, 4, 5
                        const R p = r.tab[3 * RW + ri] * pyx[k] + r.tab[4 * RW + ri] * dd;
                        r.phyx[q] = p;
                        tt = dd * r.tab[5 * RW + ri] + p;
                    }
                    r.hy[q] = hyo[k] + S * tt;
                }
            }
        }
        __syncthreads();
        // ---- E half step over the region (reads Hx, Hy, writes Ez, J, psi_E)
        R src_v = R(0);
        const R *gsrc = nullptr;
        R *gap_rec = nullptr, *rec = nullptr;
        if (MODE == 0) {
            const int n = w.n0 + t;
            src_v = src_s[t];
            gap_rec = w.gap ? w.gap + (long long)(n + 1) * Mg : nullptr;
            rec = w.rec ? w.rec + (long long)(n - w.rec0) * w.Mdi : nullptr;
        } else {
            gsrc = w.gap ? w.gap + (long long)(w.n0 - t) * Mg : nullptr;
        }
        {
            R ez[NK], hy[NK], hyL[NK], hx[NK], hxD[NK], pex[NK], pey[NK], jo[NK], ca[NK], cb[NK], bj[NK], a1[NK],
                a2[NK];
#pragma unroll
            for (int k = 0; k < NK; ++k) {
                const unsigned f = fk[k];
                const int q = q0 + k * TBY * RW;
                ez[k] = hy[k] = hyL[k] = hx[k] = hxD[k] = pex[k] = pey[k] = R(0);
                jo[k] = ca[k] = cb[k] = bj[k] = a1[k] = a2[k] = R(0);
                if (f & F_E) {
                    ez[k] = r.ez[q];
                    hy[k] = r.hy[q];
                    hyL[k] = r.hy[q - 1];
                    hx[k] = r.hx[q];
                    hxD[k] = r.hx[q - RW];
                }
                if (f & F_EXP) pex[k] = r.pezx[q];
                if (f & F_EYP) pey[k] = r.pezy[q];
                if (f & F_DRU) {
                    jo[k] = r.J[q];
                    ca[k] = r.ca[q];
                    cb[k] = r.cb[q];
                    bj[k] = r.bJ[q];
                    if (MODE == 1) {
                        a1[k] = r.a1[q];
                        a2[k] = r.a2[q];
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < NK; ++k) {
                const unsigned f = fk[k];
                if (!(f & F_E)) continue;
                const int q = q0 + k * TBY * RW, rj = ty + k * TBY, j = y0 + rj;
                const R dHy = hy[k] - hyL[k];
                const R dHx = hx[k] - hxD[k];
                R cx = dHy, cy = dHx;
                if (f & F_EXP) {  // x tables at node positions: rows 0, 1, 2
                    const R p = r.tab[0 * RW + ri] * pex[k] + r.tab[1 * RW + ri] * dHy;
                    r.pezx[q] = p;
                    cx = dHy * r.tab[2 * RW + ri] + p;
                }
                if (f & F_EYP) {  // y tables at node positions: rows 6, 7, 8
                    const R p = r.tab[6 * RW + rj] * pey[k] + r.tab[7 * RW + rj] * dHx;
                    r.pezy[q] = p;
                    cy = dHx * r.tab[8 * RW + rj] + p;
                }
                const R curl = S * (cx - cy);
                // the step kernel's e_update; records for the tile's own nodes
                const bool own = (f & F_OWN) != 0, gap = (f & F_GAP) != 0;
                const int gidx = gap ? (j - g.gy0) * g.gnx + (i - g.gx0) : 0;
                R src = R(0);
                if (MODE == 0) {
                    if (f & F_SRC) src = src_v;
                } else if (gap) {
                    src = -c.eps_g * gsrc[gidx];
                }
                R en;
                if (f & F_DRU) {
                    // drude() with its rho~-only coefficients precomputed
                    en = ca[k] * ez[k] + cb[k] * (curl - c.half1pkJ * jo[k] - src);
                    const R jn = c.kJ * jo[k] + bj[k] * (en + ez[k]);
                    R term = R(0);
                    if (MODE == 1) term = -c.t_eps * (en - ez[k]) - a1[k] * (en + ez[k]) - a2[k] * (jn + jo[k]);
                    r.J[q] = jn;
                    if (own) {
                        if (MODE == 0) {
                            if (rec) rec[(long long)(j - g.dy0) * g.dp + (i - g.dxa)] = en;
                        } else {
                            const int o = (rj - T) * tb + (ri - T);
                            r.G[o] += (double)r.rec[t * TBT * TBT + o] * (double)term;
                        }
                    }
                } else {
                    en = ez[k] + (curl - src) * (gap ? c.inv_eps_g : c.inv_eps_s);
                    if (MODE == 0 && own && (f & F_DES) && rec) rec[(long long)(j - g.dy0) * g.dp + (i - g.dxa)] = en;
                }
                if (MODE == 0 && own && gap && gap_rec) gap_rec[gidx] = en;
                r.ez[q] = en;
            }
        }
        __syncthreads();
    }

    // ---- store the tile's own nodes into the other buffer of the pair
    for (int o = flat; o < tb * tb; o += NTH) {
        const int ox = o % tb, oy = o / tb;
        const int oi = blockIdx.x * tb + ox, oj = blockIdx.y * tb + oy;
        if (oi >= nx || oj >= ny) continue;
        const int q = (oy + T) * RW + (ox + T);
        const long long gq = (long long)oj * P + oi;
        out.Ez[gq] = r.ez[q];
        out.Hx[gq] = r.hx[q];
        out.Hy[gq] = r.hy[q];
        if (in_range(oi, g.dx0, g.dnx) && in_range(oj, g.dy0, g.dny)) {
            const long long dg = (long long)(oj - g.dy0) * g.dp + (oi - g.dxa);
            out.J[dg] = r.J[q];
            if (MODE == 1) w.G[dg] = r.G[o];
        }
        if (np > 0) {
            const int se = slab_e(oi, nx, np), sh = slab_h(oi, nx, np);
            const int te = slab_e(oj, ny, np), th = slab_h(oj, ny, np);
            if (se >= 0) out.pezx[(long long)oj * np2 + se] = r.pezx[q];
            if (sh >= 0) out.phyx[(long long)oj * np2 + sh] = r.phyx[q];
            if (te >= 0) out.pezy[(long long)te * P + oi] = r.pezy[q];
            if (th >= 0) out.phxy[(long long)th * P + oi] = r.phxy[q];
        }
    }
}

}  // namespace

template <typename R>
int tb2d_max_steps()
{
    int dev = 0, smem = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    for (int T = Dim<R>::TM; T >= 1; --T) {
        const size_t b = tb2d_smem_bytes((int)sizeof(R), T);
        if (b > (size_t)smem) continue;
        if (cudaFuncSetAttribute(k_tb2d<R, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b) != cudaSuccess ||
            cudaFuncSetAttribute(k_tb2d<R, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        return T;
    }
    return 0;
}

template <typename R>
int launch_tb2d(int mode, const Geo2D &g, const State2D<R> &in, const State2D<R> &out, int coef_slot,
                const Pml1D<R> &px, const Pml1D<R> &py, const Tb2D<R> &w, cudaStream_t st)
{
    const dim3 block(Dim<R>::RW, TBY), grid((g.nx + w.tile - 1) / w.tile, (g.ny + w.tile - 1) / w.tile);
    const size_t smem = tb2d_smem_bytes((int)sizeof(R), w.count);
    if (mode == 0) k_tb2d<R, 0><<<grid, block, smem, st>>>(g, in, out, coef_slot, px, py, w);
    else k_tb2d<R, 1><<<grid, block, smem, st>>>(g, in, out, coef_slot, px, py, w);
    return 1;
}

// This translation unit's copy of the coefficient slots (constant memory is
// per translation unit).
template <typename R>
cudaError_t upload_coef_tb2d(int slot, const Coef<R> &c, cudaStream_t st)
{
    return write_coef_slot(slot, c, st);
}

template int tb2d_max_steps<float>();
template int tb2d_max_steps<double>();
template int launch_tb2d<float>(int, const Geo2D &, const State2D<float> &, const State2D<float> &, int,
                                const Pml1D<float> &, const Pml1D<float> &, const Tb2D<float> &, cudaStream_t);
template int launch_tb2d<double>(int, const Geo2D &, const State2D<double> &, const State2D<double> &, int,
                                 const Pml1D<double> &, const Pml1D<double> &, const Tb2D<double> &, cudaStream_t);
template cudaError_t upload_coef_tb2d<float>(int, const Coef<float> &, cudaStream_t);
template cudaError_t upload_coef_tb2d<double>(int, const Coef<double> &, cudaStream_t);

}  // namespace fdtd
