// Fused 2D TM_z leapfrog step (Ez, Hx, Hy, Jz + CPML) for sm_103a.
//
// One launch advances the whole grid by one time step n -> n+1: the H half
// step of mu0 dH/dt = -curl E and the E half step of Eq. (10a,b) (J and
// sigma E averaged over the step, scaled units, see Coef).  State is read
// from one buffer of a ping-pong pair and written to the other, so every
// state word crosses HBM once per step (24 B per vacuum node).
//
// Each thread owns four adjacent nodes of one row (16-byte vector loads and
// stores; rows are padded to 32 nodes), 32 x 4 threads per block, i.e. a
// 128 x 4 node tile, up to 10 blocks per SM (a block-shape sweep on the
// 2048^2 workload: 128 x 4 beat 128 x 8, 128 x 16 and 128 x 2).  A thread
// computes the new Hx and Hy of its nodes and, in registers, the new Hy left
// of its first node and the new Hx below its
// nodes, which its E updates need: 6 vector and 3 scalar loads per 4 nodes,
// neighbour rows served by L1, no exchange between threads and no barrier.
//
// Paths are chosen per block (uniform): blocks whose nodes and neighbours
// are clear of walls and CPML slabs run vector code, with per-node design /
// gap / source logic only when the tile touches those boxes; border blocks
// run a scalar path with CPML.  The design-box arrays (J, rho~, records, G)
// use the library's pitched layout: column origin dxa (a multiple of 4) and row pitch dp (a
// multiple of 4), so that they load as vectors too.  Indices are 32-bit.

#include "coef_slots.cuh"
#include "fdtd_internal.h"
#include "launch.cuh"

namespace fdtd {

namespace {

constexpr int BX = 32, BY = 4, VX = 4;
constexpr int TILE_X = BX * VX;

__device__ __forceinline__ bool in_range(int v, int lo, int n) { return (unsigned)(v - lo) < (unsigned)n; }

// Vector path for blocks none of whose read nodes (x0-1 .. x0+TILE_X,
// y0-1 .. y0+BY) is a wall or CPML node (uniform across the block).  The
// host counts blocks with the same predicate (step2d_block_counts).
__host__ __device__ __forceinline__ bool vector_tile(int nx, int ny, int np, int x0, int y0)
{
    return x0 - 1 >= np + 1 && x0 + TILE_X <= nx - np - 2 && y0 - 1 >= np + 1 && y0 + BY <= ny - np - 2;
}

// Programmatic dependent launch: the step kernels are launched with
// programmatic stream serialisation, so a step's blocks may be scheduled
// while the previous step drains; they wait here, before touching any state,
// until the previous grid has completed and its writes are visible.
__device__ __forceinline__ void wait_previous_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp(double x) { return __drcp_rn(x); }

__device__ __forceinline__ void ld4(const float *__restrict__ p, float (&o)[4])
{
    const float4 t = *reinterpret_cast<const float4 *>(p);
    o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
}
__device__ __forceinline__ void ld4(const double *__restrict__ p, double (&o)[4])
{
    const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
__device__ __forceinline__ void st4(float *p, const float (&o)[4])
{
    *reinterpret_cast<float4 *>(p) = make_float4(o[0], o[1], o[2], o[3]);
}
__device__ __forceinline__ void st4(double *p, const double (&o)[4])
{
    reinterpret_cast<double2 *>(p)[0] = make_double2(o[0], o[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(o[2], o[3]);
}

// Drude node of Eq. (10a,b): new E and J from old E, J, the scaled curl and
// the source; term = the Eq. (25a-c) bracket folded through Eq. (27).
template <typename R, int MODE>
__device__ __forceinline__ void drude(const Coef<R> &c, R rt, R ez, R jo, R curl, R src, R &en, R &jn, R &term)
{
    const R eps = c.eps_s + rt * c.d_eps;
    const R psi = c.psi_s + rt * (c.psi - c.psi_s);
    const R sig = c.sig_max * rt * (R(1) - rt);
    const R bJ = R(0.5) * psi * c.inv1g;
    const R hs = R(0.5) * (sig + bJ);
    const R cb = rcp(eps + hs);
    const R ca = (eps - hs) * cb;
    en = ca * ez + cb * (curl - c.half1pkJ * jo - src);
    jn = c.kJ * jo + bJ * (en + ez);
    if (MODE == 1)
        term = -c.t_eps * (en - ez) - c.t_sig * (R(1) - R(2) * rt) * R(0.5) * (en + ez) -
               c.t_dpsi * rcp(psi) * R(0.5) * (jn + jo);
}

// Scalar E update of one node (border blocks): design, gap and source
// logic, records and sensitivity.
template <typename R, int MODE>
__device__ __forceinline__ R e_update(const Geo2D &g, const State2D<R> &in, const State2D<R> &out, const Coef<R> &c,
                                      const Step2D<R> &a, int i, int j, R ez, R curl)
{
    const bool gap = in_range(i, g.gx0, g.gnx) && in_range(j, g.gy0, g.gny);
    const int gidx = (j - g.gy0) * g.gnx + (i - g.gx0);
    R src = R(0);
    if (MODE == 0) {
        if (in_range(i, g.sx0, g.sx1 - g.sx0) && in_range(j, g.sy0, g.sy1 - g.sy0)) src = *a.src;
    } else if (gap) {
        src = -c.eps_g * a.gap_src[gidx];
    }
    const bool des = in_range(i, g.dx0, g.dnx) && in_range(j, g.dy0, g.dny);
    const int d = (j - g.dy0) * g.dp + (i - g.dxa);
    R en;
    if (des && !gap) {
        R jn, term = R(0);
        drude<R, MODE>(c, a.rho_t[d], ez, in.J[d], curl, src, en, jn, term);
        out.J[d] = jn;
        if (MODE == 0) {
            if (a.rec) a.rec[d] = en;
        } else {
            a.G[d] += (double)a.rec[d] * (double)term;
        }
    } else {
        en = ez + (curl - src) * (gap ? c.inv_eps_g : c.inv_eps_s);
        if (MODE == 0 && des && a.rec) a.rec[d] = en;
    }
    if (MODE == 0 && gap && a.gap_rec) a.gap_rec[gidx] = en;
    return en;
}

// Scalar step of the four nodes i0 .. i0+3 of row j in a border block.
template <typename R, int MODE>
__device__ __forceinline__ void border_step(const Geo2D &g, const State2D<R> &in, const State2D<R> &out,
                                         const Coef<R> &c, const Pml1D<R> &px, const Pml1D<R> &py,
                                         const Step2D<R> &a, int i0, int j)
{
    const int nx = g.nx, ny = g.ny, np = g.npml, P = g.px;
    const R S = c.S;
    if (j >= ny) return;
    // New Hx at (ii, jj + 1/2); psi written only for the own node.
    auto hx_new = [&](int ii, int jj, bool own) -> R {
        if ((unsigned)ii >= (unsigned)nx || (unsigned)jj >= (unsigned)ny) return R(0);
        const int qq = jj * P + ii;
        const R h = in.Hx[qq];
        if (jj + 1 >= ny) return h;
        const R dd = in.Ez[qq + P] - in.Ez[qq];
        R t = dd;
        if (np > 0 && (jj < np || jj >= ny - 1 - np)) {
            const int qs = (jj < np ? jj : np + jj - (ny - 1 - np)) * P + ii;
            const R p = py.bH[jj] * in.phxy[qs] + py.cH[jj] * dd;
            if (own) out.phxy[qs] = p;
            t = dd * py.kiH[jj] + p;
        }
        return h - S * t;
    };
    // New Hy at (ii + 1/2, jj).
    auto hy_new = [&](int ii, int jj, bool own) -> R {
        if ((unsigned)ii >= (unsigned)nx || (unsigned)jj >= (unsigned)ny) return R(0);
        const int qq = jj * P + ii;
        const R h = in.Hy[qq];
        if (ii + 1 >= nx) return h;
        const R dd = in.Ez[qq + 1] - in.Ez[qq];
        R t = dd;
        if (np > 0 && (ii < np || ii >= nx - 1 - np)) {
            const int qs = jj * 2 * np + (ii < np ? ii : np + ii - (nx - 1 - np));
            const R p = px.bH[ii] * in.phyx[qs] + px.cH[ii] * dd;
            if (own) out.phyx[qs] = p;
            t = dd * px.kiH[ii] + p;
        }
        return h + S * t;
    };
    for (int k = 0; k < VX; ++k) {
        const int i = i0 + k;
        if (i >= nx) return;
        const int q = j * P + i;
        const R ez = in.Ez[q];
        const R hxn = hx_new(i, j, true);
        const R hyn = hy_new(i, j, true);
        R en = ez;
        if (i >= 1 && i <= nx - 2 && j >= 1 && j <= ny - 2) {
            const R dHy = hyn - hy_new(i - 1, j, false);
            const R dHx = hxn - hx_new(i, j - 1, false);
            R cx = dHy, cy = dHx;
            if (np > 0 && (i < np || i >= nx - np)) {
                const int qs = j * 2 * np + (i < np ? i : i - (nx - 2 * np));
                const R p = px.bE[i] * in.pezx[qs] + px.cE[i] * dHy;
                out.pezx[qs] = p;
                cx = dHy * px.kiE[i] + p;
            }
            if (np > 0 && (j < np || j >= ny - np)) {
                const int qs = (j < np ? j : j - (ny - 2 * np)) * P + i;
                const R p = py.bE[j] * in.pezy[qs] + py.cE[j] * dHx;
                out.pezy[qs] = p;
                cy = dHx * py.kiE[j] + p;
            }
            en = e_update<R, MODE>(g, in, out, c, a, i, j, ez, S * (cx - cy));
        }
        out.Ez[q] = en;
        out.Hx[q] = hxn;
        out.Hy[q] = hyn;
    }
}

template <typename R, int MODE>
__device__ __forceinline__ void step2d_body(const Geo2D &g, const State2D<R> &in, const State2D<R> &out,
                                            const Coef<R> &c, const Pml1D<R> &px, const Pml1D<R> &py,
                                            const Step2D<R> &a, int bx, int by)
{
    const int x0 = bx * TILE_X, y0 = by * BY;
    const int i0 = x0 + threadIdx.x * VX, j = y0 + threadIdx.y;
    const int nx = g.nx, ny = g.ny, np = g.npml, P = g.px;
    const R S = c.S;

    if (vector_tile(nx, ny, np, x0, y0)) {
        const int q = j * P + i0;
        R e[4], eN[4], eS[4], hx[4], hxS[4], hy[4];
        ld4(in.Ez + q, e);
        ld4(in.Ez + q + P, eN);
        ld4(in.Ez + q - P, eS);
        ld4(in.Hx + q, hx);
        ld4(in.Hx + q - P, hxS);
        ld4(in.Hy + q, hy);
        const R ezW = in.Ez[q - 1], ezE = in.Ez[q + VX], hyW = in.Hy[q - 1];
        R hxn[4], yn[5], curlS[4];
        yn[0] = hyW + S * (e[0] - ezW);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            hxn[k] = hx[k] - S * (eN[k] - e[k]);
            const R hxsn = hxS[k] - S * (e[k] - eS[k]);
            yn[k + 1] = hy[k] + S * ((k < 3 ? e[k + 1] : ezE) - e[k]);
            curlS[k] = -(hxn[k] - hxsn);
        }
        R en[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) curlS[k] += yn[k + 1] - yn[k];

        const bool touches = (x0 < g.dx0 + g.dnx && x0 + TILE_X > g.dx0 && y0 < g.dy0 + g.dny && y0 + BY > g.dy0) ||
                             (MODE == 0 && x0 < g.sx1 && x0 + TILE_X > g.sx0 && y0 < g.sy1 && y0 + BY > g.sy0);
        if (!touches) {
            const R Se = S * c.inv_eps_s;
#pragma unroll
            for (int k = 0; k < 4; ++k) en[k] = e[k] + Se * curlS[k];
        } else {
            // Design / gap / source tile: vector loads of the design arrays
            // when this thread's four nodes lie in the pitched design rows.
            const bool rdes = in_range(j, g.dy0, g.dny);
            const bool vdes = rdes && in_range(i0, g.dxa, g.dp);
            const int d0 = (j - g.dy0) * g.dp + (i0 - g.dxa);
            R J4[4] = {R(0), R(0), R(0), R(0)}, rt4[4] = {R(0), R(0), R(0), R(0)}, em4[4] = {R(0), R(0), R(0), R(0)};
            if (vdes) {
                ld4(in.J + d0, J4);
                ld4(a.rho_t + d0, rt4);
                if (MODE == 1) ld4(a.rec + d0, em4);
            }
            const bool rgap = in_range(j, g.gy0, g.gny);
            const bool rsrc = MODE == 0 && in_range(j, g.sy0, g.sy1 - g.sy0);
            R jn4[4];
            double gadd[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int i = i0 + k;
                const R curl = S * curlS[k];
                const bool gap = rgap && in_range(i, g.gx0, g.gnx);
                const int gidx = (j - g.gy0) * g.gnx + (i - g.gx0);
                R src = R(0);
                if (MODE == 0) {
                    if (rsrc && in_range(i, g.sx0, g.sx1 - g.sx0)) src = *a.src;
                } else if (gap) {
                    src = -c.eps_g * a.gap_src[gidx];
                }
                jn4[k] = J4[k];
                gadd[k] = 0.0;
                if (vdes && in_range(i, g.dx0, g.dnx) && !gap) {
                    R term = R(0);
                    drude<R, MODE>(c, rt4[k], e[k], J4[k], curl, src, en[k], jn4[k], term);
                    if (MODE == 1) gadd[k] = (double)em4[k] * (double)term;
                } else {
                    en[k] = e[k] + (curl - src) * (gap ? c.inv_eps_g : c.inv_eps_s);
                }
                if (MODE == 0 && gap && a.gap_rec) a.gap_rec[gidx] = en[k];
            }
            if (vdes) {
                st4(out.J + d0, jn4);
                if (MODE == 0) {
                    if (a.rec) st4(a.rec + d0, en);
                } else {
                    double G4[4];
                    ld4(a.G + d0, G4);
#pragma unroll
                    for (int k = 0; k < 4; ++k) G4[k] += gadd[k];
                    st4(a.G + d0, G4);
                }
            }
        }
        st4(out.Ez + q, en);
        st4(out.Hx + q, hxn);
        const R hy4[4] = {yn[1], yn[2], yn[3], yn[4]};
        st4(out.Hy + q, hy4);
        return;
    }

    border_step<R, MODE>(g, in, out, c, px, py, a, i0, j);
}

template <typename R, int MODE>
__global__ void __launch_bounds__(BX *BY, 10)
    k_step2d(const __grid_constant__ Geo2D g, const __grid_constant__ State2D<R> in,
             const __grid_constant__ State2D<R> out, int slot,
             const __grid_constant__ Pml1D<R> px, const __grid_constant__ Pml1D<R> py,
             const __grid_constant__ Step2D<R> a)
{
    wait_previous_grid();
    step2d_body<R, MODE>(g, in, out, coef_at<R>(slot), px, py, a, blockIdx.x, blockIdx.y);
}

// One forward (recompute) step and one adjoint step of independent states in
// one launch: blocks with blockIdx.z == 0 advance the forward state, those
// with blockIdx.z == 1 the adjoint state.
template <typename R>
__global__ void __launch_bounds__(BX *BY, 10)
    k_step2d_pair(const __grid_constant__ Geo2D g, const __grid_constant__ State2D<R> fin,
                  const __grid_constant__ State2D<R> fout, const __grid_constant__ Step2D<R> fa,
                  const __grid_constant__ State2D<R> ain, const __grid_constant__ State2D<R> aout,
                  const __grid_constant__ Step2D<R> aa, int slot,
                  const __grid_constant__ Pml1D<R> px, const __grid_constant__ Pml1D<R> py)
{
    wait_previous_grid();
    if (blockIdx.z == 0) step2d_body<R, 0>(g, fin, fout, coef_at<R>(slot), px, py, fa, blockIdx.x, blockIdx.y);
    else step2d_body<R, 1>(g, ain, aout, coef_at<R>(slot), px, py, aa, blockIdx.x, blockIdx.y);
}

}  // namespace

void step2d_block_counts(const Geo2D &g, long long *total, long long *vector)
{
    const int gx = (g.nx + TILE_X - 1) / TILE_X, gy = (g.ny + BY - 1) / BY;
    long long v = 0;
    for (int by = 0; by < gy; ++by)
        for (int bx = 0; bx < gx; ++bx) v += vector_tile(g.nx, g.ny, g.npml, bx * TILE_X, by * BY) ? 1 : 0;
    *total = (long long)gx * gy;
    *vector = v;
}

template <typename R>
int launch_step2d(int mode, const Geo2D &g, const State2D<R> &in, const State2D<R> &out, int c,
                  const Pml1D<R> &px, const Pml1D<R> &py, const Step2D<R> &a, cudaStream_t st,
                  const cudaAccessPolicyWindow *win)
{
    dim3 grid((g.nx + TILE_X - 1) / TILE_X, (g.ny + BY - 1) / BY), block(BX, BY);
    if (mode == 0) launch_pdl_win(k_step2d<R, 0>, grid, block, st, win, g, in, out, c, px, py, a);
    else launch_pdl_win(k_step2d<R, 1>, grid, block, st, win, g, in, out, c, px, py, a);
    return 1;
}

template <typename R>
int launch_step2d_pair(const Geo2D &g, const State2D<R> &fin, const State2D<R> &fout, const Step2D<R> &fa,
                       const State2D<R> &ain, const State2D<R> &aout, const Step2D<R> &aa, int c,
                       const Pml1D<R> &px, const Pml1D<R> &py, cudaStream_t st, const cudaAccessPolicyWindow *win)
{
    dim3 grid((g.nx + TILE_X - 1) / TILE_X, (g.ny + BY - 1) / BY, 2), block(BX, BY);
    launch_pdl_win(k_step2d_pair<R>, grid, block, st, win, g, fin, fout, fa, ain, aout, aa, c, px, py);
    return 1;
}

template int launch_step2d_pair<float>(const Geo2D &, const State2D<float> &, const State2D<float> &,
                                       const Step2D<float> &, const State2D<float> &, const State2D<float> &,
                                       const Step2D<float> &, int, const Pml1D<float> &,
                                       const Pml1D<float> &, cudaStream_t, const cudaAccessPolicyWindow *);
template int launch_step2d_pair<double>(const Geo2D &, const State2D<double> &, const State2D<double> &,
                                        const Step2D<double> &, const State2D<double> &, const State2D<double> &,
                                        const Step2D<double> &, int, const Pml1D<double> &,
                                        const Pml1D<double> &, cudaStream_t, const cudaAccessPolicyWindow *);
template int launch_step2d<float>(int, const Geo2D &, const State2D<float> &, const State2D<float> &,
                                  int, const Pml1D<float> &, const Pml1D<float> &,
                                  const Step2D<float> &, cudaStream_t, const cudaAccessPolicyWindow *);
template int launch_step2d<double>(int, const Geo2D &, const State2D<double> &, const State2D<double> &,
                                   int, const Pml1D<double> &, const Pml1D<double> &,
                                   const Step2D<double> &, cudaStream_t, const cudaAccessPolicyWindow *);

}  // namespace fdtd

namespace fdtd {
template <typename R>
cudaError_t upload_coef_2d(int slot, const Coef<R> &c, cudaStream_t st)
{
    return write_coef_slot(slot, c, st);
}
template cudaError_t upload_coef_2d<float>(int, const Coef<float> &, cudaStream_t);
template cudaError_t upload_coef_2d<double>(int, const Coef<double> &, cudaStream_t);
}  // namespace fdtd
