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
// slab of its axis.  Each thread owns four x-adjacent nodes (32 x 8 x 4-node
// blocks): where those nodes and their halo are clear of walls and CPML it
// runs vector code with the curls written out, elsewhere generic per-node
// code with CPML.
//
// Every E component of a node inside the design box takes the material of
// rho~ at that node (Eq. 5); the adjoint sums the Eq. (25) brackets of the
// three components into the node's FP64 accumulator.
#include <utility>

#include "fdtd_internal.h"

namespace fdtd {

namespace {

// Tiles: 8 x 8 x 4 threads, four x-adjacent nodes each, i.e.
// 32 x 8 x 4 nodes (a warp reads 128 contiguous bytes per row).
constexpr int VX = 4, TBX = 8, TBY = 8, TBZ = 4;
constexpr int TX = TBX * VX;

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

// Are the four nodes i0 .. i0+3 of row (j, k) and their one-node halo clear
// of walls and CPML slabs?
__device__ __forceinline__ bool thread_interior(const Geo3D &g, int i0, int j, int k)
{
    const int np = g.npml;
    return i0 - 1 >= np + 1 && i0 + VX <= g.n[0] - np - 2 && j - 1 >= np + 1 && j + 1 <= g.n[1] - np - 2 &&
           k - 1 >= np + 1 && k + 1 <= g.n[2] - np - 2;
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

// Generic H update of node (i, j, k): every component, CPML where needed.
template <typename R>
__device__ __forceinline__ void h_node(const Geo3D &g, const State3D<R> &s, const Coef<R> &c, const Pml3D<R> &pm,
                                       int i, int j, int k)
{
    const int p[3] = {i, j, k};
    const long long st[3] = {1, g.px, g.PP};
    const long long q = k * g.PP + (long long)j * g.px + i;
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
        const int a = (cc + 1) % 3, b = (cc + 2) % 3;
        // H component cc exists where the node is not on the last plane of a or b.
        if (p[a] > g.n[a] - 2 || p[b] > g.n[b] - 2) continue;
        const R da = s.E[b][q + st[a]] - s.E[b][q];  // d_a E_b (forward)
        const R db = s.E[a][q + st[b]] - s.E[a][q];  // d_b E_a
        R ta = da * pm.kiH[a][p[a]], tb = db * pm.kiH[b][p[b]];
        const int sa = slabH(p[a], g.n[a], g.npml), sb = slabH(p[b], g.n[b], g.npml);
        if (sa >= 0) {
            R &ps = s.ph[cc][0][pidx(g, a, sa, i, j, k)];
            ps = pm.bH[a][p[a]] * ps + pm.cH[a][p[a]] * da;
            ta += ps;
        }
        if (sb >= 0) {
            R &ps = s.ph[cc][1][pidx(g, b, sb, i, j, k)];
            ps = pm.bH[b][p[b]] * ps + pm.cH[b][p[b]] * db;
            tb += ps;
        }
        s.H[cc][q] -= c.S * (ta - tb);
    }
}

// Generic E (and J) update of node (i, j, k): every component, CPML where
// needed, design / gap / source logic, records and sensitivity.
template <typename R, int MODE>
__device__ __forceinline__ void e_node(const Geo3D &g, const State3D<R> &s, const Coef<R> &c, const Pml3D<R> &pm,
                                       const Step3D<R> &a3, int i, int j, int k)
{
    const int p[3] = {i, j, k};
    const long long st[3] = {1, g.px, g.PP};
    const long long q = k * g.PP + (long long)j * g.px + i;
    const bool gap = in_range(i, g.g0[0], g.gn[0]) && in_range(j, g.g0[1], g.gn[1]) && in_range(k, g.g0[2], g.gn[2]);
    const int gidx = ((k - g.g0[2]) * g.gn[1] + (j - g.g0[1])) * g.gn[0] + (i - g.g0[0]);
    const bool des = in_range(i, g.d0[0], g.dn[0]) && in_range(j, g.d0[1], g.dn[1]) && in_range(k, g.d0[2], g.dn[2]);
    const long long d = ((long long)(k - g.d0[2]) * g.dn[1] + (j - g.d0[1])) * g.dp + (i - g.dxa);
    const bool src_node = MODE == 0 && in_range(i, g.s0[0], g.s1[0] - g.s0[0]) &&
                          in_range(j, g.s0[1], g.s1[1] - g.s0[1]) && in_range(k, g.s0[2], g.s1[2] - g.s0[2]);
    const R eps_bg = gap ? c.eps_g : (k < g.sub_hi ? c.eps_sub : c.eps_s);
    R rt = R(0);
    if (des && !gap) rt = a3.rho_t[d];
    double gsum = 0.0;
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
        const int a = (cc + 1) % 3, b = (cc + 2) % 3;
        // E component cc is updated away from the walls: 0 < p < n-1 across,
        // p <= n-2 along its own axis.
        if (p[cc] > g.n[cc] - 2 || p[a] < 1 || p[a] > g.n[a] - 2 || p[b] < 1 || p[b] > g.n[b] - 2) continue;
        const R da = s.H[b][q] - s.H[b][q - st[a]];  // d_a H_b (backward)
        const R db = s.H[a][q] - s.H[a][q - st[b]];  // d_b H_a
        R ta = da * pm.kiE[a][p[a]], tb = db * pm.kiE[b][p[b]];
        const int sa = slabE(p[a], g.n[a], g.npml), sb = slabE(p[b], g.n[b], g.npml);
        if (sa >= 0) {
            R &ps = s.pe[cc][0][pidx(g, a, sa, i, j, k)];
            ps = pm.bE[a][p[a]] * ps + pm.cE[a][p[a]] * da;
            ta += ps;
        }
        if (sb >= 0) {
            R &ps = s.pe[cc][1][pidx(g, b, sb, i, j, k)];
            ps = pm.bE[b][p[b]] * ps + pm.cE[b][p[b]] * db;
            tb += ps;
        }
        const R curl = c.S * (ta - tb);
        R src = R(0);
        if (MODE == 0) {
            if (src_node && cc == g.src_comp) src = *a3.src;
        } else if (gap) {
            src = -c.eps_g * a3.gap_src[(long long)cc * g.Mg + gidx];
        }
        const R e = s.E[cc][q];
        R en;
        if (des && !gap) {
            const R eps = c.eps_s + rt * c.d_eps;
            const R psi = c.psi_s + rt * (c.psi - c.psi_s);
            const R sig = c.sig_max * rt * (R(1) - rt);
            const R bJ = R(0.5) * psi * c.inv1g;
            const R hs = R(0.5) * (sig + bJ);
            const R cb = rcp(eps + hs);
            const R ca = (eps - hs) * cb;
            const R jo = s.J[cc][d];
            en = ca * e + cb * (curl - c.half1pkJ * jo - src);
            const R jn = c.kJ * jo + bJ * (en + e);
            s.J[cc][d] = jn;
            if (MODE == 0) {
                if (a3.rec) a3.rec[(long long)cc * g.Mdi + d] = en;
            } else {
                // Eq. (25a-c) folded through the chain rule of Eq. (27).
                const R term = -c.d_eps * (en - e) - c.sig_max * (R(1) - R(2) * rt) * R(0.5) * (en + e) -
                               (c.psi - c.psi_s) * rcp(psi) * R(0.5) * (jn + jo);
                gsum += (double)a3.rec[(long long)cc * g.Mdi + d] * (double)term;
            }
        } else {
            en = e + (curl - src) * rcp(eps_bg);
            if (MODE == 0 && des && a3.rec) a3.rec[(long long)cc * g.Mdi + d] = en;
        }
        s.E[cc][q] = en;
        if (MODE == 0 && gap && a3.gap_rec) a3.gap_rec[(long long)cc * g.Mg + gidx] = en;
    }
    if (MODE == 1 && des && !gap) a3.G[d] += gsum;
}

// Interior H half step: curl E with forward differences, no CPML.
//   Hx -= S (dy Ez - dz Ey),  Hy -= S (dz Ex - dx Ez),  Hz -= S (dx Ey - dy Ex)
template <typename R>
__global__ void __launch_bounds__(TBX *TBY *TBZ) k_h3d_in(Geo3D g, State3D<R> s, Coef<R> c, Pml3D<R> pm)
{
    wait_previous_grid();
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TBY, z0 = blockIdx.z * TBZ;
    const int i0 = x0 + threadIdx.x * VX, j = y0 + threadIdx.y, k = z0 + threadIdx.z;
    if (j >= g.n[1] || k >= g.n[2]) return;
    if (!thread_interior(g, i0, j, k)) {
        for (int v = 0; v < VX; ++v)
            if (i0 + v < g.n[0]) h_node<R>(g, s, c, pm, i0 + v, j, k);
        return;
    }
    const long long q = k * g.PP + (long long)j * g.px + i0;
    const long long P = g.px, PP = g.PP;
    R ex[4], exN[4], exU[4], ey[4], eyU[4], ez[4], ezN[4], hx[4], hy[4], hz[4];
    ld4(s.E[0] + q, ex);
    ld4(s.E[0] + q + P, exN);
    ld4(s.E[0] + q + PP, exU);
    ld4(s.E[1] + q, ey);
    ld4(s.E[1] + q + PP, eyU);
    ld4(s.E[2] + q, ez);
    ld4(s.E[2] + q + P, ezN);
    ld4(s.H[0] + q, hx);
    ld4(s.H[1] + q, hy);
    ld4(s.H[2] + q, hz);
    const R eyE = s.E[1][q + VX], ezE = s.E[2][q + VX];
    const R S = c.S;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const R ezx = v < 3 ? ez[v + 1] : ezE, eyx = v < 3 ? ey[v + 1] : eyE;
        hx[v] -= S * ((ezN[v] - ez[v]) - (eyU[v] - ey[v]));
        hy[v] -= S * ((exU[v] - ex[v]) - (ezx - ez[v]));
        hz[v] -= S * ((eyx - ey[v]) - (exN[v] - ex[v]));
    }
    st4(s.H[0] + q, hx);
    st4(s.H[1] + q, hy);
    st4(s.H[2] + q, hz);
}

// Interior E half step: curl H with backward differences, no CPML; per
// component the Drude update of Eq. (10a,b) in the design box.
//   curl_x = dy Hz - dz Hy,  curl_y = dz Hx - dx Hz,  curl_z = dx Hy - dy Hx
template <typename R, int MODE>
__global__ void __launch_bounds__(TBX *TBY *TBZ)
    k_e3d_in(Geo3D g, State3D<R> s, Coef<R> c, Pml3D<R> pm, Step3D<R> a3)
{
    wait_previous_grid();
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TBY, z0 = blockIdx.z * TBZ;
    const int i0 = x0 + threadIdx.x * VX, j = y0 + threadIdx.y, k = z0 + threadIdx.z;
    if (j >= g.n[1] || k >= g.n[2]) return;
    if (!thread_interior(g, i0, j, k)) {
        for (int v = 0; v < VX; ++v)
            if (i0 + v < g.n[0]) e_node<R, MODE>(g, s, c, pm, a3, i0 + v, j, k);
        return;
    }
    const long long q = k * g.PP + (long long)j * g.px + i0;
    const long long P = g.px, PP = g.PP;
    R hx[4], hxS[4], hxD[4], hy[4], hyD[4], hz[4], hzS[4];
    ld4(s.H[0] + q, hx);
    ld4(s.H[0] + q - P, hxS);
    ld4(s.H[0] + q - PP, hxD);
    ld4(s.H[1] + q, hy);
    ld4(s.H[1] + q - PP, hyD);
    ld4(s.H[2] + q, hz);
    ld4(s.H[2] + q - P, hzS);
    const R hyW = s.H[1][q - 1], hzW = s.H[2][q - 1];
    R curl[3][4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const R hyx = v > 0 ? hy[v - 1] : hyW, hzx = v > 0 ? hz[v - 1] : hzW;
        curl[0][v] = c.S * ((hz[v] - hzS[v]) - (hy[v] - hyD[v]));
        curl[1][v] = c.S * ((hx[v] - hxD[v]) - (hz[v] - hzx));
        curl[2][v] = c.S * ((hy[v] - hyx) - (hx[v] - hxS[v]));
    }
    const bool touches = (x0 < g.d0[0] + g.dn[0] && x0 + TX > g.d0[0] && y0 < g.d0[1] + g.dn[1] &&
                          y0 + TBY > g.d0[1] && z0 < g.d0[2] + g.dn[2] && z0 + TBZ > g.d0[2]) ||
                         (MODE == 0 && x0 < g.s1[0] && x0 + TX > g.s0[0] && y0 < g.s1[1] && y0 + TBY > g.s0[1] &&
                          z0 < g.s1[2] && z0 + TBZ > g.s0[2]);
    const R inv_bg = rcp(k < g.sub_hi ? c.eps_sub : c.eps_s);
    if (!touches) {
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
            R e[4];
            ld4(s.E[cc] + q, e);
#pragma unroll
            for (int v = 0; v < 4; ++v) e[v] += curl[cc][v] * inv_bg;
            st4(s.E[cc] + q, e);
        }
        return;
    }
    // Design / gap / source tile.
    const bool rdes = in_range(j, g.d0[1], g.dn[1]) && in_range(k, g.d0[2], g.dn[2]);
    const bool vdes = rdes && in_range(i0, g.dxa, g.dp);
    const long long d0 = ((long long)(k - g.d0[2]) * g.dn[1] + (j - g.d0[1])) * g.dp + (i0 - g.dxa);
    const bool rgap = in_range(j, g.g0[1], g.gn[1]) && in_range(k, g.g0[2], g.gn[2]);
    const bool rsrc = MODE == 0 && in_range(j, g.s0[1], g.s1[1] - g.s0[1]) && in_range(k, g.s0[2], g.s1[2] - g.s0[2]);
    R rt4[4] = {R(0), R(0), R(0), R(0)};
    if (vdes) ld4(a3.rho_t + d0, rt4);
    double gadd[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
        R e[4], J4[4] = {R(0), R(0), R(0), R(0)}, em4[4] = {R(0), R(0), R(0), R(0)};
        ld4(s.E[cc] + q, e);
        if (vdes) {
            ld4(s.J[cc] + d0, J4);
            if (MODE == 1) ld4(a3.rec + cc * g.Mdi + d0, em4);
        }
        R en[4], jn4[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int i = i0 + v;
            const bool gap = rgap && in_range(i, g.g0[0], g.gn[0]);
            const int gidx = ((k - g.g0[2]) * g.gn[1] + (j - g.g0[1])) * g.gn[0] + (i - g.g0[0]);
            R src = R(0);
            if (MODE == 0) {
                if (rsrc && cc == g.src_comp && in_range(i, g.s0[0], g.s1[0] - g.s0[0])) src = *a3.src;
            } else if (gap) {
                src = -c.eps_g * a3.gap_src[(long long)cc * g.Mg + gidx];
            }
            jn4[v] = J4[v];
            if (vdes && in_range(i, g.d0[0], g.dn[0]) && !gap) {
                const R rt = rt4[v];
                const R eps = c.eps_s + rt * c.d_eps;
                const R psi = c.psi_s + rt * (c.psi - c.psi_s);
                const R sig = c.sig_max * rt * (R(1) - rt);
                const R bJ = R(0.5) * psi * c.inv1g;
                const R hs = R(0.5) * (sig + bJ);
                const R cb = rcp(eps + hs);
                const R ca = (eps - hs) * cb;
                en[v] = ca * e[v] + cb * (curl[cc][v] - c.half1pkJ * J4[v] - src);
                jn4[v] = c.kJ * J4[v] + bJ * (en[v] + e[v]);
                if (MODE == 1) {
                    // Eq. (25a-c) folded through the chain rule of Eq. (27).
                    const R term = -c.d_eps * (en[v] - e[v]) -
                                   c.sig_max * (R(1) - R(2) * rt) * R(0.5) * (en[v] + e[v]) -
                                   (c.psi - c.psi_s) * rcp(psi) * R(0.5) * (jn4[v] + J4[v]);
                    gadd[v] += (double)em4[v] * (double)term;
                }
            } else {
                en[v] = e[v] + (curl[cc][v] - src) * (gap ? rcp(c.eps_g) : inv_bg);
            }
            if (MODE == 0 && gap && a3.gap_rec) a3.gap_rec[(long long)cc * g.Mg + gidx] = en[v];
        }
        st4(s.E[cc] + q, en);
        if (vdes) {
            st4(s.J[cc] + d0, jn4);
            if (MODE == 0 && a3.rec) st4(a3.rec + cc * g.Mdi + d0, en);
        }
    }
    if (MODE == 1 && vdes) {
        double G4[4];
        ld4(a3.G + d0, G4);
#pragma unroll
        for (int v = 0; v < 4; ++v) G4[v] += gadd[v];
        st4(a3.G + d0, G4);
    }
}

}  // namespace

template <typename... KArgs, typename... Args>
void launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

template <typename R>
int launch_step3d(int mode, const Geo3D &g, const State3D<R> &s, const Coef<R> &c, const Pml3D<R> &pm,
                  const Step3D<R> &a, cudaStream_t st)
{
    dim3 vblock(TBX, TBY, TBZ), vgrid((g.n[0] + TX - 1) / TX, (g.n[1] + TBY - 1) / TBY, (g.n[2] + TBZ - 1) / TBZ);
    launch_pdl(k_h3d_in<R>, vgrid, vblock, st, g, s, c, pm);
    if (mode == 0) launch_pdl(k_e3d_in<R, 0>, vgrid, vblock, st, g, s, c, pm, a);
    else launch_pdl(k_e3d_in<R, 1>, vgrid, vblock, st, g, s, c, pm, a);
    return 2;
}

template int launch_step3d<float>(int, const Geo3D &, const State3D<float> &, const Coef<float> &,
                                  const Pml3D<float> &, const Step3D<float> &, cudaStream_t);
template int launch_step3d<double>(int, const Geo3D &, const State3D<double> &, const Coef<double> &,
                                   const Pml3D<double> &, const Step3D<double> &, cudaStream_t);

}  // namespace fdtd
