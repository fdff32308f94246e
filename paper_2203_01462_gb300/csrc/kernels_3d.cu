// 3D Yee leapfrog (Ex, Ey, Ez, Hx, Hy, Hz + Drude Jx, Jy, Jz + CPML) for sm_103a.
//
// Node (i, j, k) carries Ex at (i+1/2, j, k), Ey at (i, j+1/2, k), Ez at
// (i, j, k+1/2), Hx at (i, j+1/2, k+1/2), Hy at (i+1/2, j, k+1/2) and Hz at
// (i+1/2, j+1/2, k); tangential E vanishes on the outer faces (PEC walls
// behind the CPML).  Two launches per step, each updating its fields in
// place: the H half step of mu0 dH/dt = -curl E, then the E half step of
// Eq. (10a,b) per component (J and sigma E averaged over the step, scaled
// units, see Coef).  Curl component c uses the cyclic axes a = c+1, b = c+2:
// curl_c = d_a F_b - d_b F_a, each derivative with its own CPML term in the
// slab of its axis.  Each thread owns four x-adjacent nodes (32 x 8 x 2-node
// blocks) and runs one vector code path everywhere: next to the PEC walls
// it skips the neighbour loads that fall outside the grid and masks the
// components that are not updated there (H_c exists where p <= n-2 along
// both of its derivative axes; E_c is updated where p <= n-2 along c and
// 1 <= p <= n-2 across), so no warp diverges into per-node code.  The CPML
// terms of a y- or z-slab are uniform over the four nodes and their psi
// arrays are x-contiguous, so they move as vectors; x-slab terms are taken
// per node.
//
// Every E component of a node inside the design box takes the material of
// rho~ at that node (Eq. 5); the adjoint sums the Eq. (25) brackets of the
// three components into the node's FP64 accumulator.

#include <algorithm>

#include "coef_slots.cuh"
#include "fdtd_internal.h"
#include "launch.cuh"

namespace fdtd {

namespace {

// Tiles: 8 x 8 x 2 threads, four x-adjacent nodes each, i.e.
// 32 x 8 x 2 nodes (a warp reads 128 contiguous bytes per row).  Shapes
// (at 768 threads per SM): 8x8x4 at 3 / 8x8x2 at 6 / 4x8x4 at 6 / 8x4x2 at
// 12 per SM; 8x8x2 and 4x8x4 were fastest, by 3-5 %.  Blocks per SM in
// FP32 (the register budget): H 6 (80 registers), forward E 7 (72), adjoint
// E 6 (80).  With the CPML terms taken one axis at a time the kernels need
// about 100 registers unbounded (128-136 with all six psi pairs held), so
// these bounds spill little (16-44 B; 148 B in the adjoint E).  256^3
// forward step: 5 blocks everywhere 242.6 us, 6 everywhere 229.3, H and
// forward E at 7 227.4, everything at 7 227.4 (adjoint 465 against 457 at
// 6), H at 7 with E at 6 231.7.
constexpr int VX = 4, TBX = 8, TBY = 8, TBZ = 2;
constexpr int TX = TBX * VX;
static_assert(WAVE3D_TX == TX && WAVE3D_TY == TBY && WAVE3D_TZ == TBZ, "wavefront tiles are the step tiles");

__device__ __forceinline__ bool in_range(int v, int lo, int n) { return (unsigned)(v - lo) < (unsigned)n; }

// Programmatic dependent launch (as in the 2D kernels): wait, before touching
// any state, until the previous grid in the stream has completed.
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
// Loads for the persistent wavefront kernel, which reads fields other blocks
// of the same launch wrote: plain (coherent) global loads, never the
// read-only path that `const __restrict__` pointers allow.
__device__ __forceinline__ void ld4c(const float *p, float (&o)[4])
{
    const float4 t = *reinterpret_cast<const float4 *>(p);
    o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
}
__device__ __forceinline__ void ld4c(const double *p, double (&o)[4])
{
    const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
template <bool COH, typename R>
__device__ __forceinline__ void ldv(const R *p, R (&o)[4])
{
    if constexpr (COH) ld4c(p, o);
    else ld4(p, o);
}

// Roundings of the plain curl update fixed, so that the half-step kernels
// and the wavefront kernel (other code around the same arithmetic) give the
// same bits: the scaled curl is rounded, then subtracted (H) or added with
// one fused multiply-add by 1/eps (E).
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rn_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double rn_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float rn_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rn_fma(double a, double b, double c) { return __fma_rn(a, b, c); }

// Plane-wave face corrections with their rounding fixed (one fused
// multiply-add, the E-face product rounded first), so that the half-step
// kernels and the wavefront kernel give the same bits.
__device__ __forceinline__ float tf_fma(float a, float b, float x) { return __fmaf_rn(a, b, x); }
__device__ __forceinline__ double tf_fma(double a, double b, double x) { return __fma_rn(a, b, x); }
__device__ __forceinline__ float tf_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double tf_mul(double a, double b) { return __dmul_rn(a, b); }

template <typename R>
__device__ __forceinline__ void zero4(R (&o)[4])
{
    o[0] = o[1] = o[2] = o[3] = R(0);
}

// Slab index of position p along an axis of n nodes (E: node positions,
// H: half positions), or -1 outside the absorbing layer.
__device__ __forceinline__ int slabE(int p, int n, int np) { return p < np ? p : (p >= n - np ? p - (n - 2 * np) : -1); }
__device__ __forceinline__ int slabH(int p, int n, int np)
{
    return p < np ? p : ((p >= n - 1 - np && p < n - 1) ? np + p - (n - 1 - np) : -1);
}

// Element of the CPML array of a slab along axis ax at slab index s and node (i, j, k).
__device__ __forceinline__ long long pidx(const Geo3D &g, int ax, int s, int i, int j, int k)
{
    const int np2 = 2 * g.npml;
    if (ax == 0) return ((long long)k * g.n[1] + j) * np2 + s;
    if (ax == 1) return ((long long)k * np2 + s) * g.px + i;
    return ((long long)s * g.n[1] + j) * g.px + i;
}

// CPML-corrected curl of four x-adjacent nodes (i0 .. i0+3, row j, plane k),
// one axis at a time.  Component c takes the derivative d[c][0] along
// a = c+1 and d[c][1] along b = c+2 (cyclic), so the two terms along axis
// ax are (c, h) = ((ax+2) % 3, 0) and ((ax+1) % 3, 1).  Each term becomes
// t = d / kappa, plus, in the slab of its axis, psi <- b psi + c d and
// t += psi; the caller forms S (t_a - t_b).  Along y and z the slab index
// and coefficients are those of row j / plane k, and the psi arrays of y-
// and z-slabs are x-contiguous, so psi moves as one vector; along x both
// are taken per node.  The kernels load the psi pair of one axis (the
// first slab axis in the order z, y, x: the only one on a face of the
// absorbing shell) before their field loads, so that both round trips
// overlap; the pairs of further axes (edges and corners of the shell) are
// loaded where they are used.  Only one pair is held across the field
// loads, not all six.
template <bool HALF>
__device__ __forceinline__ void slab_x(const Geo3D &g, int i0, int (&sx)[4])
{
#pragma unroll
    for (int v = 0; v < 4; ++v)  // nodes past the last one are row padding: no slab
        sx[v] = i0 + v >= g.n[0] ? -1 : (HALF ? slabH(i0 + v, g.n[0], g.npml) : slabE(i0 + v, g.n[0], g.npml));
}

template <typename R, bool COH, int AX>
__device__ __forceinline__ void cpml_load_axis(const Geo3D &g, R *const (&psi)[3][2], int i0, int j, int k, int sy,
                                               int sz, const int (&sx)[4], R (&p)[2][4])
{
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int c = (AX + 2 - h) % 3;
        zero4(p[h]);
        if (AX == 0) {
#pragma unroll
            for (int v = 0; v < 4; ++v)
                if (sx[v] >= 0) p[h][v] = psi[c][h][pidx(g, 0, sx[v], i0 + v, j, k)];
        } else if (AX == 1) {
            if (sy >= 0) ldv<COH>(psi[c][h] + pidx(g, 1, sy, i0, j, k), p[h]);
        } else {
            if (sz >= 0) ldv<COH>(psi[c][h] + pidx(g, 2, sz, i0, j, k), p[h]);
        }
    }
}

// The early load: the pair of axis pa (2, 1 or 0).
template <typename R, bool COH>
__device__ __forceinline__ void cpml_preload(const Geo3D &g, R *const (&psi)[3][2], int pa, int i0, int j, int k,
                                             int sy, int sz, const int (&sx)[4], R (&p)[2][4])
{
    if (pa == 2) cpml_load_axis<R, COH, 2>(g, psi, i0, j, k, sy, sz, sx, p);
    else if (pa == 1) cpml_load_axis<R, COH, 1>(g, psi, i0, j, k, sy, sz, sx, p);
    else cpml_load_axis<R, COH, 0>(g, psi, i0, j, k, sy, sz, sx, p);
}

// Axis AX: d[c][h] <- d / kappa (+ the updated psi in the slab of AX) for
// its two terms, psi stored back.  pre: the pair loaded early when pa == AX.
template <typename R, bool COH, int AX>
__device__ __forceinline__ void cpml_axis(const Geo3D &g, R *const (&psi)[3][2], const R *const (&tb)[3],
                                          const R *const (&tc)[3], const R *const (&tk)[3], int i0, int j, int k,
                                          int sy, int sz, const int (&sx)[4], int pa, const R (&pre)[2][4],
                                          R (&d)[3][2][4])
{
    // with kappa = 1 everywhere the 1/kappa tables are not read (the product
    // by 1 is exact, so the result is the same); coefficient tables are
    // read-only: non-coherent loads, free to move past stores
    const bool k1 = g.kappa1 != 0;
    R kk[4];
#pragma unroll
    for (int v = 0; v < 4; ++v)
        kk[v] = AX == 0 ? ((!k1 && i0 + v < g.n[0]) ? __ldg(tk[0] + i0 + v) : R(1))
                        : (k1 ? R(1) : __ldg(tk[AX] + (AX == 1 ? j : k)));
    const bool any = AX == 0 ? (sx[0] >= 0 || sx[1] >= 0 || sx[2] >= 0 || sx[3] >= 0) : (AX == 1 ? sy >= 0 : sz >= 0);
    if (!any) {
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int v = 0; v < 4; ++v) d[(AX + 2 - h) % 3][h][v] = d[(AX + 2 - h) % 3][h][v] * kk[v];
        return;
    }
    R ps[2][4];
    if (pa == AX) {
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int v = 0; v < 4; ++v) ps[h][v] = pre[h][v];
    } else {
        cpml_load_axis<R, COH, AX>(g, psi, i0, j, k, sy, sz, sx, ps);
    }
    R bb[4], cc[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        if (AX == 0) {
            bb[v] = sx[v] >= 0 ? __ldg(tb[0] + i0 + v) : R(0);
            cc[v] = sx[v] >= 0 ? __ldg(tc[0] + i0 + v) : R(0);
        } else {
            bb[v] = __ldg(tb[AX] + (AX == 1 ? j : k));
            cc[v] = __ldg(tc[AX] + (AX == 1 ? j : k));
        }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int c = (AX + 2 - h) % 3;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const R dd = d[c][h][v];
            R t = dd * kk[v];
            if (AX != 0 || sx[v] >= 0) {
                ps[h][v] = bb[v] * ps[h][v] + cc[v] * dd;
                t += ps[h][v];
            }
            d[c][h][v] = t;
        }
        if (AX == 0) {
#pragma unroll
            for (int v = 0; v < 4; ++v)
                if (sx[v] >= 0) psi[c][h][pidx(g, 0, sx[v], i0 + v, j, k)] = ps[h][v];
        } else {
            st4(psi[c][h] + pidx(g, AX, AX == 1 ? sy : sz, i0, j, k), ps[h]);
        }
    }
}

// All three axes (z, y, x), then out[c] = S (t_a - t_b).
template <typename R, bool COH>
__device__ __forceinline__ void cpml_curl(const Geo3D &g, R *const (&psi)[3][2], const R *const (&tb)[3],
                                          const R *const (&tc)[3], const R *const (&tk)[3], int i0, int j, int k,
                                          int sy, int sz, const int (&sx)[4], int pa, const R (&pre)[2][4], R S,
                                          R (&d)[3][2][4], R (&out)[3][4])
{
    cpml_axis<R, COH, 2>(g, psi, tb, tc, tk, i0, j, k, sy, sz, sx, pa, pre, d);
    cpml_axis<R, COH, 1>(g, psi, tb, tc, tk, i0, j, k, sy, sz, sx, pa, pre, d);
    cpml_axis<R, COH, 0>(g, psi, tb, tc, tk, i0, j, k, sy, sz, sx, pa, pre, d);
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int v = 0; v < 4; ++v) out[c][v] = rn_mul(S, d[c][0][v] - d[c][1][v]);
}

// H half step, four x-adjacent nodes per thread:
//   Hx -= S (dy Ez - dz Ey),  Hy -= S (dz Ex - dx Ez),  Hz -= S (dx Ey - dy Ex)
// (forward differences).  Threads clear of every CPML slab run the plain
// update; the others add the CPML terms (cpml_curl).
// One tile (bx, by, bz) of the H half step.  COH: loads for the wavefront
// kernel; FOLD: inc (may then be null) is the plane wave's incident row of
// this step, whose face corrections are added before the stores.
template <typename R, bool COH, bool FOLD>
__device__ __forceinline__ void h_tile(const Geo3D &g, const State3D<R> &s, const Coef<R> &c, const Pml3D<R> &pm,
                                       int bx, int by, int bz, const R *inc)
{
    const int i0 = (bx * TBX + threadIdx.x) * VX, j = by * TBY + threadIdx.y, k = bz * TBZ + threadIdx.z;
    const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
    if (i0 >= n0 || j >= n1 || k >= n2) return;
    const long long q = k * g.PP + (long long)j * g.px + i0;
    const long long P = g.px, PP = g.PP;
    const bool yin = j <= n1 - 2, zin = k <= n2 - 2, xin = i0 + VX <= n0 - 1;  // next row / plane / node exist
    const int np = g.npml;
    const int sy = slabH(j, n1, np), sz = slabH(k, n2, np);
    const bool xslab = i0 < np || i0 + VX - 1 >= n0 - 1 - np;
    const bool pml = xslab || sy >= 0 || sz >= 0;
    int sx[4], pa = 0;
    R pre[2][4];
    if (pml) {
        slab_x<true>(g, i0, sx);
        pa = sz >= 0 ? 2 : (sy >= 0 ? 1 : 0);
        cpml_preload<R, COH>(g, s.ph, pa, i0, j, k, sy, sz, sx, pre);
    }
    R ex[4], exN[4], exU[4], ey[4], eyU[4], ez[4], ezN[4], hx[4], hy[4], hz[4];
    ldv<COH>(s.E[0] + q, ex);
    ldv<COH>(s.E[1] + q, ey);
    ldv<COH>(s.E[2] + q, ez);
    if (yin) {
        ldv<COH>(s.E[0] + q + P, exN);
        ldv<COH>(s.E[2] + q + P, ezN);
    } else {
        zero4(exN);
        zero4(ezN);
    }
    if (zin) {
        ldv<COH>(s.E[0] + q + PP, exU);
        ldv<COH>(s.E[1] + q + PP, eyU);
    } else {
        zero4(exU);
        zero4(eyU);
    }
    ldv<COH>(s.H[0] + q, hx);
    ldv<COH>(s.H[1] + q, hy);
    ldv<COH>(s.H[2] + q, hz);
    const R eyE = xin ? s.E[1][q + VX] : R(0), ezE = xin ? s.E[2][q + VX] : R(0);
    const R S = c.S;
    R cu[3][4];
    if (!pml) {
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const R ezx = v < 3 ? ez[v + 1] : ezE, eyx = v < 3 ? ey[v + 1] : eyE;
            cu[0][v] = rn_mul(S, (ezN[v] - ez[v]) - (eyU[v] - ey[v]));
            cu[1][v] = rn_mul(S, (exU[v] - ex[v]) - (ezx - ez[v]));
            cu[2][v] = rn_mul(S, (eyx - ey[v]) - (exN[v] - ex[v]));
        }
    } else {
        R d[3][2][4];  // d[c][0]: along c+1, d[c][1]: along c+2 (forward differences of E)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            d[0][0][v] = ezN[v] - ez[v];                         // d_y Ez
            d[0][1][v] = eyU[v] - ey[v];                         // d_z Ey
            d[1][0][v] = exU[v] - ex[v];                         // d_z Ex
            d[1][1][v] = (v < 3 ? ez[v + 1] : ezE) - ez[v];      // d_x Ez
            d[2][0][v] = (v < 3 ? ey[v + 1] : eyE) - ey[v];      // d_x Ey
            d[2][1][v] = exN[v] - ex[v];                         // d_y Ex
        }
        cpml_curl<R, COH>(g, s.ph, pm.bH, pm.cH, pm.kiH, i0, j, k, sy, sz, sx, pa, pre, S, d, cu);
    }
    if (xin && yin && zin) {
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            hx[v] = rn_sub(hx[v], cu[0][v]);
            hy[v] = rn_sub(hy[v], cu[1][v]);
            hz[v] = rn_sub(hz[v], cu[2][v]);
        }
    } else {
        // last row / plane / node: H_x exists where j, k <= n-2, H_y where
        // k, i <= n-2, H_z where i, j <= n-2 (nodes past n0 are padding)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int i = i0 + v;
            if (yin && zin && i < n0) hx[v] = rn_sub(hx[v], cu[0][v]);
            if (zin && i <= n0 - 2) hy[v] = rn_sub(hy[v], cu[1][v]);
            if (yin && i <= n0 - 2) hz[v] = rn_sub(hz[v], cu[2][v]);
        }
    }
    if constexpr (FOLD) {
        if (inc) {
            // the H-face corrections of the plane wave (see the TFSF notes)
            const int lx = g.tf_lo[0], ly = g.tf_lo[1], lz = g.tf_lo[2];
            const int ux = g.tf_hi[0], uy = g.tf_hi[1], uz = g.tf_hi[2];
            if ((k == lz - 1 || k == uz) && j >= ly && j <= uy) {
                const R a = k == uz ? -S : S, e = k == uz ? inc[uz - lz] : inc[0];
#pragma unroll
                for (int v = 0; v < 4; ++v)
                    if (i0 + v >= lx && i0 + v < ux) hy[v] = tf_fma(a, e, hy[v]);
            }
            if ((j == ly - 1 || j == uy) && k >= lz && k <= uz) {
                const R a = j == uy ? S : -S, e = inc[k - lz];
#pragma unroll
                for (int v = 0; v < 4; ++v)
                    if (i0 + v >= lx && i0 + v < ux) hz[v] = tf_fma(a, e, hz[v]);
            }
        }
    }
    st4(s.H[0] + q, hx);
    st4(s.H[1] + q, hy);
    st4(s.H[2] + q, hz);
}

// The H half step of the whole grid, bottom up or (zrev) top down; FOLD:
// with the plane wave's H-face corrections of incident row inc.
template <typename R, bool FOLD>
__global__ void __launch_bounds__(TBX *TBY *TBZ, sizeof(R) == 4 ? 6 : 1)
    k_h3d(Geo3D g, State3D<R> s, int slot, Pml3D<R> pm, int zrev, const R *inc)
{
    wait_previous_grid();
    const int bz = zrev ? gridDim.z - 1 - blockIdx.z : blockIdx.z;
    h_tile<R, false, FOLD>(g, s, coef_at<R>(slot), pm, blockIdx.x, blockIdx.y, bz, inc);
}

// E half step: curl H with backward differences (CPML terms as in the H
// kernel); per component the Drude update of Eq. (10a,b) in the design box.
//   curl_x = dy Hz - dz Hy,  curl_y = dz Hx - dx Hz,  curl_z = dx Hy - dy Hx
// One tile (bx, by, bz) of the E half step.  COH: loads for the wavefront
// kernel; FOLD (forward): the plane wave's face corrections of row
// a3.tf_inc (when set) added before the stores.
template <typename R, int MODE, bool COH, bool FOLD>
__device__ __forceinline__ void e_tile(const Geo3D &g, const State3D<R> &s, const Coef<R> &c, const Pml3D<R> &pm,
                                       const Step3D<R> &a3, int bx, int by, int bz)
{
    const int x0 = bx * TX, y0 = by * TBY, z0 = bz * TBZ;
    const int i0 = x0 + threadIdx.x * VX, j = y0 + threadIdx.y, k = z0 + threadIdx.z;
    const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
    if (i0 >= n0 || j >= n1 || k >= n2) return;
    const long long q = k * g.PP + (long long)j * g.px + i0;
    const long long P = g.px, PP = g.PP;
    const int np = g.npml;
    const int sy = slabE(j, n1, np), sz = slabE(k, n2, np);
    const bool xslab = i0 < np || i0 + VX - 1 >= n0 - np;
    const bool pml = xslab || sy >= 0 || sz >= 0;
    int sx[4], pa = 0;
    R pre[2][4];
    if (pml) {
        slab_x<false>(g, i0, sx);
        pa = sz >= 0 ? 2 : (sy >= 0 ? 1 : 0);
        cpml_preload<R, COH>(g, s.pe, pa, i0, j, k, sy, sz, sx, pre);
    }
    R hx[4], hxS[4], hxD[4], hy[4], hyD[4], hz[4], hzS[4], e[3][4];
    ldv<COH>(s.H[0] + q, hx);
    ldv<COH>(s.H[1] + q, hy);
    ldv<COH>(s.H[2] + q, hz);
    if (j >= 1) {
        ldv<COH>(s.H[0] + q - P, hxS);
        ldv<COH>(s.H[2] + q - P, hzS);
    } else {
        zero4(hxS);
        zero4(hzS);
    }
    if (k >= 1) {
        ldv<COH>(s.H[0] + q - PP, hxD);
        ldv<COH>(s.H[1] + q - PP, hyD);
    } else {
        zero4(hxD);
        zero4(hyD);
    }
    const R hyW = i0 >= 1 ? s.H[1][q - 1] : R(0), hzW = i0 >= 1 ? s.H[2][q - 1] : R(0);
    // all E loads before any store (the compiler cannot reorder them past
    // stores through other field pointers)
    ldv<COH>(s.E[0] + q, e[0]);
    ldv<COH>(s.E[1] + q, e[1]);
    ldv<COH>(s.E[2] + q, e[2]);
    R curl[3][4];
    if (!pml) {
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const R hyx = v > 0 ? hy[v - 1] : hyW, hzx = v > 0 ? hz[v - 1] : hzW;
            curl[0][v] = rn_mul(c.S, (hz[v] - hzS[v]) - (hy[v] - hyD[v]));
            curl[1][v] = rn_mul(c.S, (hx[v] - hxD[v]) - (hz[v] - hzx));
            curl[2][v] = rn_mul(c.S, (hy[v] - hyx) - (hx[v] - hxS[v]));
        }
    } else {
        R d[3][2][4];  // backward differences of H
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            d[0][0][v] = hz[v] - hzS[v];                         // d_y Hz
            d[0][1][v] = hy[v] - hyD[v];                         // d_z Hy
            d[1][0][v] = hx[v] - hxD[v];                         // d_z Hx
            d[1][1][v] = hz[v] - (v > 0 ? hz[v - 1] : hzW);      // d_x Hz
            d[2][0][v] = hy[v] - (v > 0 ? hy[v - 1] : hyW);      // d_x Hy
            d[2][1][v] = hx[v] - hxS[v];                         // d_y Hx
        }
        cpml_curl<R, COH>(g, s.pe, pm.bE, pm.cE, pm.kiE, i0, j, k, sy, sz, sx, pa, pre, c.S, d, curl);
    }
    // E_c is updated where p <= n-2 along c and 1 <= p <= n-2 across; a
    // component that is not updated keeps its value (zero on the walls).
    const bool full = i0 >= 1 && i0 + VX <= n0 - 1 && j >= 1 && j <= n1 - 2 && k >= 1 && k <= n2 - 2;
    const bool jmid = j >= 1 && j <= n1 - 2, kmid = k >= 1 && k <= n2 - 2;
    auto upd = [&](int cc, int v) -> bool {
        const int i = i0 + v;
        const bool imid = i >= 1 && i <= n0 - 2;
        if (cc == 0) return i <= n0 - 2 && jmid && kmid;
        if (cc == 1) return j <= n1 - 2 && imid && kmid;
        return k <= n2 - 2 && imid && jmid;
    };
    const bool touches = (x0 < g.d0[0] + g.dn[0] && x0 + TX > g.d0[0] && y0 < g.d0[1] + g.dn[1] &&
                          y0 + TBY > g.d0[1] && z0 < g.d0[2] + g.dn[2] && z0 + TBZ > g.d0[2]) ||
                         (MODE == 0 && x0 < g.s1[0] && x0 + TX > g.s0[0] && y0 < g.s1[1] && y0 + TBY > g.s0[1] &&
                          z0 < g.s1[2] && z0 + TBZ > g.s0[2]);
    const R inv_bg = rcp(k < g.sub_hi ? c.eps_sub : c.eps_s);
    // the E-face corrections of the plane wave (see the TFSF notes; the
    // faces lie in background material)
    auto tf_fix = [&](int cc, R(&x)[4]) {
        if constexpr (FOLD && MODE == 0) {
            if (!a3.tf_inc) return;
            const int lx = g.tf_lo[0], ly = g.tf_lo[1], lz = g.tf_lo[2];
            const int ux = g.tf_hi[0], uy = g.tf_hi[1], uz = g.tf_hi[2];
            const R *hi = a3.tf_inc + (uz - lz + 1);
            if (cc == 0 && (k == lz || k == uz) && j >= ly && j <= uy) {
                const R m = tf_mul(k == uz ? -c.S : c.S, k == uz ? hi[uz - lz + 1] : hi[0]);
#pragma unroll
                for (int v = 0; v < 4; ++v)
                    if (i0 + v >= lx && i0 + v < ux) x[v] = tf_fma(m, inv_bg, x[v]);
            }
            if (cc == 2 && j >= ly && j <= uy && k >= lz && k < uz) {
#pragma unroll
                for (int v = 0; v < 4; ++v)
                    if (i0 + v == lx || i0 + v == ux)
                        x[v] = tf_fma(tf_mul(i0 + v == ux ? c.S : -c.S, hi[k - lz + 1]), inv_bg, x[v]);
            }
        }
    };
    if (!touches) {
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
#pragma unroll
            for (int v = 0; v < 4; ++v)
                if (full || upd(cc, v)) e[cc][v] = rn_fma(curl[cc][v], inv_bg, e[cc][v]);
            tf_fix(cc, e[cc]);
            st4(s.E[cc] + q, e[cc]);
        }
        return;
    }
    // Design / gap / source tile: every design-array load first, then the
    // per-node updates, then the stores.
    const bool rdes = in_range(j, g.d0[1], g.dn[1]) && in_range(k, g.d0[2], g.dn[2]);
    const bool vdes = rdes && in_range(i0, g.dxa, g.dp);
    const long long d0 = ((long long)(k - g.d0[2]) * g.dn[1] + (j - g.d0[1])) * g.dp + (i0 - g.dxa);
    const bool rgap = in_range(j, g.g0[1], g.gn[1]) && in_range(k, g.g0[2], g.gn[2]);
    const bool rsrc = MODE == 0 && in_range(j, g.s0[1], g.s1[1] - g.s0[1]) && in_range(k, g.s0[2], g.s1[2] - g.s0[2]);
    R rt4[4] = {R(0), R(0), R(0), R(0)}, J4[3][4], em4[3][4];
    double G4[4] = {0.0, 0.0, 0.0, 0.0}, gadd[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int cc = 0; cc < 3; ++cc)
#pragma unroll
        for (int v = 0; v < 4; ++v) J4[cc][v] = em4[cc][v] = R(0);
    if (vdes) {
        ld4(a3.rho_t + d0, rt4);
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
            ldv<COH>(s.J[cc] + d0, J4[cc]);
            if (MODE == 1) ldv<COH>(a3.rec + cc * g.Mdi + d0, em4[cc]);
        }
        if (MODE == 1) ldv<COH>(a3.G + d0, G4);
    }
    const R src_fwd = (MODE == 0 && rsrc) ? *a3.src : R(0);
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
        R en[4], jn4[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int i = i0 + v;
            const bool gap = rgap && in_range(i, g.g0[0], g.gn[0]);
            const int gidx = ((k - g.g0[2]) * g.gn[1] + (j - g.g0[1])) * g.gn[0] + (i - g.g0[0]);
            R src = R(0);
            if (MODE == 0) {
                if (rsrc && cc == g.src_comp && in_range(i, g.s0[0], g.s1[0] - g.s0[0])) src = src_fwd;
            } else if (gap) {
                src = -c.eps_g * a3.gap_src[(long long)cc * g.Mg + gidx];
            }
            jn4[v] = J4[cc][v];
            if (!full && !upd(cc, v)) {
                en[v] = e[cc][v];
            } else if (vdes && in_range(i, g.d0[0], g.dn[0]) && !gap) {
                const R rt = rt4[v];
                const R eps = c.eps_s + rt * c.d_eps;
                const R psi = c.psi_s + rt * (c.psi - c.psi_s);
                const R sig = c.sig_max * rt * (R(1) - rt);
                const R bJ = R(0.5) * psi * c.inv1g;
                const R hs = R(0.5) * (sig + bJ);
                const R cb = rcp(eps + hs);
                const R ca = (eps - hs) * cb;
                en[v] = ca * e[cc][v] + cb * (curl[cc][v] - c.half1pkJ * J4[cc][v] - src);
                jn4[v] = c.kJ * J4[cc][v] + bJ * (en[v] + e[cc][v]);
                if (MODE == 1) {
                    // Eq. (25a-c) folded through the chain rule of Eq. (27).
                    const R term = -c.t_eps * (en[v] - e[cc][v]) -
                                   c.t_sig * (R(1) - R(2) * rt) * R(0.5) * (en[v] + e[cc][v]) -
                                   c.t_dpsi * rcp(psi) * R(0.5) * (jn4[v] + J4[cc][v]);
                    gadd[v] += (double)em4[cc][v] * (double)term;
                }
            } else {
                en[v] = rn_fma(curl[cc][v] - src, gap ? rcp(c.eps_g) : inv_bg, e[cc][v]);
            }
            if (MODE == 0 && gap && a3.gap_rec && (full || upd(cc, v)))
                a3.gap_rec[(long long)cc * g.Mg + gidx] = en[v];
        }
        tf_fix(cc, en);
        st4(s.E[cc] + q, en);
        if (vdes) {
            st4(s.J[cc] + d0, jn4);
            if (MODE == 0 && a3.rec) st4(a3.rec + cc * g.Mdi + d0, en);
        }
    }
    if (MODE == 1 && vdes) {
#pragma unroll
        for (int v = 0; v < 4; ++v) G4[v] += gadd[v];
        st4(a3.G + d0, G4);
    }
}

template <typename R, int MODE, bool FOLD>
__global__ void __launch_bounds__(TBX *TBY *TBZ, sizeof(R) == 4 ? (MODE == 1 ? 6 : 7) : 1)
    k_e3d(Geo3D g, State3D<R> s, int slot, Pml3D<R> pm, Step3D<R> a3, int zrev)
{
    wait_previous_grid();
    const int bz = zrev ? gridDim.z - 1 - blockIdx.z : blockIdx.z;
    e_tile<R, MODE, false, FOLD>(g, s, coef_at<R>(slot), pm, a3, blockIdx.x, blockIdx.y, bz);
}

// ------------------------------------------------ plane wave (TFSF notes)
//
// An x-polarised plane wave along +z enters through the faces of the
// total-field box: components whose Yee position lies in the closed box
// [tf_lo, tf_hi] hold the total field, the others the scattered field.  A
// curl that reaches across the box boundary needs the incident value of the
// component on the other side; only E_x and H_y carry one.  The faces lie in
// background material (the box encloses the design box, away from the
// CPML), where each half step is E += S curl / eps or H -= S curl, so the
// half-step kernels add the correction to the updated value before storing
// it (h_tile / e_tile with FOLD):
//   H_y(i, j, lo_z - 1) += S Ei(lo_z)     H_y(i, j, hi_z) -= S Ei(hi_z)
//   H_z(i, lo_y - 1, k) -= S Ei(k)        H_z(i, hi_y, k) += S Ei(k)
//   E_x(i, j, lo_z) += S Hi(lo_z - 1) / eps(lo_z)
//   E_x(i, j, hi_z) -= S Hi(hi_z) / eps(hi_z)
//   E_z(lo_x, j, k) -= S Hi(k) / eps(k)   E_z(hi_x, j, k) += S Hi(k) / eps(k)
// with i in [lo_x, hi_x), j in [lo_y, hi_y], k in [lo_z, hi_z] (H_z) or
// [lo_z, hi_z) (E_z).  Ei = E_x^n and Hi = H_y^{n+1/2} of the incident column.

// The incident column: E_x(k) at z = k and H_y(k) at z = k + 1/2 of a
// laterally uniform field, updated exactly as the 3D kernels update those
// components (x and y derivatives zero): H_y -= S t_z, E_x += (S (0 - t_z) -
// J) / eps, t_z the kappa-scaled z difference plus its CPML term.  One block;
// two barriers per step.
template <typename R>
__global__ void __launch_bounds__(256) k_tfsf_column(Geo3D g, Pml3D<R> pm, R S, R eps_s, R eps_sub,
                                                     const R *__restrict__ src, int nsteps, R *col, R *tab)
{
    const int nz = g.n[2], np = g.npml, lz = g.tf_lo[2], Lz = g.tf_hi[2] - lz + 1, row = 2 * Lz + 1;
    R *E = col, *H = col + nz, *pE = col + 2 * nz, *pH = col + 3 * nz;
    for (int k = threadIdx.x; k < 4 * nz; k += blockDim.x) col[k] = R(0);
    const R inv_s = rcp(eps_s), inv_sub = rcp(eps_sub);
    __syncthreads();
    for (int n = 0; n < nsteps; ++n) {
        R *out = tab + (long long)n * row;
        for (int q = threadIdx.x; q < Lz; q += blockDim.x) out[q] = E[lz + q];
        for (int k = threadIdx.x; k <= nz - 2; k += blockDim.x) {
            const R d = E[k + 1] - E[k];
            R tz = d * pm.kiH[2][k];
            if (slabH(k, nz, np) >= 0) {
                pH[k] = pm.bH[2][k] * pH[k] + pm.cH[2][k] * d;
                tz += pH[k];
            }
            H[k] -= S * tz;
        }
        __syncthreads();
        for (int q = threadIdx.x; q <= Lz; q += blockDim.x) out[Lz + q] = H[lz - 1 + q];
        const R J = src[n];
        for (int k = 1 + threadIdx.x; k <= nz - 2; k += blockDim.x) {
            const R d = H[k] - H[k - 1];
            R tz = d * pm.kiE[2][k];
            if (slabE(k, nz, np) >= 0) {
                pE[k] = pm.bE[2][k] * pE[k] + pm.cE[2][k] * d;
                tz += pE[k];
            }
            const R curl = S * (R(0) - tz);
            const R js = (k >= g.s0[2] && k < g.s1[2]) ? J : R(0);
            E[k] += (curl - js) * (k < g.sub_hi ? inv_sub : inv_s);
        }
        __syncthreads();
    }
}

// ------------------------------------------------ wavefront: several steps per launch
//
// k_wave3d runs `count` steps in one persistent launch whose blocks are all
// resident (cooperative launch).  The half steps are cut into jobs (one
// phase on one z slab of two planes) and items (up to tpi x-adjacent tiles
// of one row of a job); block b takes items b, b + G, b + 2G, ... of the
// job list (G blocks), whose order puts every job after the jobs it
// depends on:
//   E_t(s) reads H_t of slabs s and s-1 (backward differences) and
//          overwrites E that H_t(s), H_t(s-1) read;
//   H_t(s) reads E_{t-1} of slabs s and s+1 (forward differences) and
//          overwrites H that E_{t-1}(s), E_{t-1}(s+1) read.
// Before an item, one thread waits (acquire loads, bounded) until the
// per-slab counters of finished items show those jobs complete; after it,
// the block's stores are fenced and the slab's counter incremented.  Since a
// block only ever waits for items earlier in the list, and the earliest
// unfinished item's block is running it, the launch always progresses.
// Each node sees exactly the arithmetic of the split launches (the plane
// wave's face corrections are added before the stores, with the same
// rounding), so the results are bit-identical; what changes is that the E
// half step of a slab runs while the H it reads is still in L2, and with
// count > 1 the next steps re-use the slab before it leaves L2.

#ifndef WAVE_MINB
#define WAVE_MINB 4
#endif

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Bounded wait until *p >= want (counts modulo 2^32).
__device__ bool wait_count(const unsigned *p, unsigned want, unsigned *abort_word, unsigned *err, long long limit)
{
    if ((int)(ld_acquire(p) - want) >= 0) return true;
    const long long t0 = clock64();
    for (;;) {
        __nanosleep(32);
        if ((int)(ld_acquire(p) - want) >= 0) return true;
        if (ld_acquire(abort_word)) return false;
        if (clock64() - t0 > limit) {
            atomicOr(err, ERR_TIMEOUT);
            atomicExch(abort_word, 1u);
            return false;
        }
    }
}

template <typename R, int MODE>
__global__ void __launch_bounds__(TBX *TBY *TBZ, sizeof(R) == 4 ? WAVE_MINB : 1)
    k_wave3d(Geo3D g, State3D<R> s, int slot, Pml3D<R> pm, Step3D<R> a0, Wave3D<R> w, unsigned *err,
             long long limit)
{
    const Coef<R> &c = coef_at<R>(slot);
    const bool lead = threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0;
    __shared__ int go;
    if (lead) go = ld_acquire(w.cnt + 2 * w.nslab) == 0u;
    __syncthreads();
    if (!go) return;
    const int nitems = 2 * w.count * w.nslab * w.ips;  // below 2^31 (checked by the host)
#pragma unroll 1
    for (int q = blockIdx.x; q < nitems; q += gridDim.x) {
        const int job = q / w.ips, r = q - job * w.ips;
        const int code = __ldg(w.jobs + job);
        const int p = code >> 16, sl = code & 0xffff, t = p >> 1;
        const bool isE = (p & 1) != 0;
        if (lead) {
            unsigned *cH = w.cnt, *cE = w.cnt + w.nslab, *abort_word = w.cnt + 2 * w.nslab;
            bool ok = true;
            if (isE) {
                const unsigned want = (unsigned)(t + 1) * (unsigned)w.ips;
                ok = wait_count(cH + sl, want, abort_word, err, limit) &&
                     (sl == 0 || wait_count(cH + sl - 1, want, abort_word, err, limit));
            } else if (t > 0) {
                const unsigned want = (unsigned)t * (unsigned)w.ips;
                ok = wait_count(cE + sl, want, abort_word, err, limit) &&
                     (sl + 1 == w.nslab || wait_count(cE + sl + 1, want, abort_word, err, limit));
            }
            go = ok;
        }
        __syncthreads();
        if (!go) return;
        const int by = r / w.ipr, bx0 = (r - by * w.ipr) * w.tpi, bx1 = min(w.gx, bx0 + w.tpi);
        if (!isE) {
            const R *inc = (MODE == 0 && w.tf) ? w.tf + (long long)(w.n0 + t) * w.tf_row : nullptr;
#pragma unroll 1
            for (int bx = bx0; bx < bx1; ++bx) h_tile<R, true, true>(g, s, c, pm, bx, by, sl, inc);
        } else {
            Step3D<R> a = a0;
            if (MODE == 0) {
                const int n = w.n0 + t;
                a.src = w.src + n;
                a.gap_rec = w.gap ? w.gap + (long long)(n + 1) * 3 * g.Mg : nullptr;
                a.rec = w.rec ? w.rec + (long long)(n - w.rec0) * 3 * g.Mdi : nullptr;
                a.tf_inc = w.tf ? w.tf + (long long)n * w.tf_row : nullptr;
            } else {
                const int m = w.n0 - t;
                a.gap_src = w.gap ? w.gap + (long long)m * 3 * g.Mg : nullptr;
                a.rec = w.rec + (long long)(m - 1 - w.rec0) * 3 * g.Mdi;
            }
#pragma unroll 1
            for (int bx = bx0; bx < bx1; ++bx) e_tile<R, MODE, true, true>(g, s, c, pm, a, bx, by, sl);
        }
        __syncthreads();
        // E items of the last step have no reader in this launch
        if (lead && (!isE || t + 1 < w.count)) {
            __threadfence();
            atomicAdd(w.cnt + (isE ? w.nslab : 0) + sl, 1u);
        }
    }
    // The last block to finish clears the counters for the next launch.
    __shared__ int last;
    if (lead) {
        __threadfence();
        last = atomicAdd(w.cnt + 2 * w.nslab + 1, 1u) + 1 == gridDim.x;
    }
    __syncthreads();
    if (last) {
        __threadfence();
        const int nt = TBX * TBY * TBZ, tid = threadIdx.x + TBX * (threadIdx.y + TBY * threadIdx.z);
        for (int i = tid; i < 2 * w.nslab; i += nt) w.cnt[i] = 0u;
        if (lead) w.cnt[2 * w.nslab + 1] = 0u;
    }
}

}  // namespace

template <typename R>
void launch_tfsf_column(const Geo3D &g, const Pml3D<R> &pm, R S, R eps_s, R eps_sub, const R *src, int nsteps,
                        R *col, R *tab, cudaStream_t st)
{
    k_tfsf_column<R><<<1, 256, 0, st>>>(g, pm, S, eps_s, eps_sub, src, nsteps, col, tab);
}

template void launch_tfsf_column<float>(const Geo3D &, const Pml3D<float> &, float, float, float, const float *,
                                        int, float *, float *, cudaStream_t);
template void launch_tfsf_column<double>(const Geo3D &, const Pml3D<double> &, double, double, double,
                                         const double *, int, double *, double *, cudaStream_t);

template <typename R>
int launch_step3d(int mode, const Geo3D &g, const State3D<R> &s, int c, const Pml3D<R> &pm,
                  const Step3D<R> &a, cudaStream_t st)
{
    dim3 vblock(TBX, TBY, TBZ), vgrid((g.n[0] + TX - 1) / TX, (g.n[1] + TBY - 1) / TBY, (g.n[2] + TBZ - 1) / TBZ);
    // The H half step sweeps the planes upwards and the E half step
    // downwards (blocks start in blockIdx order), so each launch begins where
    // the previous one ended, on planes whose fields are still in L2.  Each
    // kernel reads only fields it does not write, so the order changes no
    // result.  A forward step of a plane wave adds the face corrections
    // inside the same launches.
    if (mode == 0 && a.tf_inc) {
        launch_pdl(k_h3d<R, true>, vgrid, vblock, st, g, s, c, pm, 0, a.tf_inc);
        launch_pdl(k_e3d<R, 0, true>, vgrid, vblock, st, g, s, c, pm, a, 1);
    } else {
        launch_pdl(k_h3d<R, false>, vgrid, vblock, st, g, s, c, pm, 0, (const R *)nullptr);
        if (mode == 0) launch_pdl(k_e3d<R, 0, false>, vgrid, vblock, st, g, s, c, pm, a, 1);
        else launch_pdl(k_e3d<R, 1, false>, vgrid, vblock, st, g, s, c, pm, a, 1);
    }
    return 2;
}


std::vector<int> wave3d_jobs(int nslab, int count, int lag)
{
    std::vector<int> jobs;
    const int phases = 2 * count;
    jobs.reserve((size_t)phases * nslab);
    for (int key = 0; key < nslab + lag * (phases - 1); ++key)
        for (int p = 0; p < phases; ++p) {
            const int sl = key - lag * p;
            if (sl >= 0 && sl < nslab) jobs.push_back(p << 16 | sl);
        }
    return jobs;
}

template <typename R>
int wave3d_blocks(int mode)
{
    int dev = 0, sms = 0, coop = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) {
        cudaGetLastError();
        return 0;
    }
    const cudaError_t e = mode == 0 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_wave3d<R, 0>, TBX * TBY * TBZ, 0)
                                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_wave3d<R, 1>, TBX * TBY * TBZ, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per * sms;
}

template <typename R>
int launch_wave3d(int mode, const Geo3D &g, const State3D<R> &s, int c, const Pml3D<R> &pm, const Step3D<R> &a0,
                  const Wave3D<R> &w, int blocks, unsigned *err, long long limit, cudaStream_t st)
{
    const long long nitems = 2LL * w.count * w.nslab * w.ips;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)std::min<long long>(blocks, nitems));
    cfg.blockDim = dim3(TBX, TBY, TBZ);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (mode == 0) cudaLaunchKernelEx(&cfg, k_wave3d<R, 0>, g, s, c, pm, a0, w, err, limit);
    else cudaLaunchKernelEx(&cfg, k_wave3d<R, 1>, g, s, c, pm, a0, w, err, limit);
    return 1;
}

template int wave3d_blocks<float>(int);
template int wave3d_blocks<double>(int);
template int launch_wave3d<float>(int, const Geo3D &, const State3D<float> &, int, const Pml3D<float> &,
                                  const Step3D<float> &, const Wave3D<float> &, int, unsigned *, long long,
                                  cudaStream_t);
template int launch_wave3d<double>(int, const Geo3D &, const State3D<double> &, int, const Pml3D<double> &,
                                   const Step3D<double> &, const Wave3D<double> &, int, unsigned *, long long,
                                   cudaStream_t);

template int launch_step3d<float>(int, const Geo3D &, const State3D<float> &, int,
                                  const Pml3D<float> &, const Step3D<float> &, cudaStream_t);
template int launch_step3d<double>(int, const Geo3D &, const State3D<double> &, int,
                                   const Pml3D<double> &, const Step3D<double> &, cudaStream_t);

}  // namespace fdtd

namespace fdtd {
template <typename R>
cudaError_t upload_coef_3d(int slot, const Coef<R> &c, cudaStream_t st)
{
    return write_coef_slot(slot, c, st);
}
template cudaError_t upload_coef_3d<float>(int, const Coef<float> &, cudaStream_t);
template cudaError_t upload_coef_3d<double>(int, const Coef<double> &, cudaStream_t);
}  // namespace fdtd
