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
// slab of its axis.  One thread per node, threads consecutive along x.
//
// Every E component of a node inside the design box takes the material of
// rho~ at that node (Eq. 5); the adjoint sums the Eq. (25) brackets of the
// three components into the node's FP64 accumulator.
#include "fdtd_internal.h"

namespace fdtd {

namespace {

constexpr int BX = 32, BY = 4, BZ = 2;

__device__ __forceinline__ bool in_range(int v, int lo, int n) { return (unsigned)(v - lo) < (unsigned)n; }
__device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp(double x) { return __drcp_rn(x); }

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

template <typename R>
__global__ void __launch_bounds__(BX *BY *BZ) k_h3d(Geo3D g, State3D<R> s, Coef<R> c, Pml3D<R> pm)
{
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    const int k = blockIdx.z * BZ + threadIdx.z;
    if (i >= g.n[0] || j >= g.n[1] || k >= g.n[2]) return;
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

template <typename R, int MODE>
__global__ void __launch_bounds__(BX *BY *BZ) k_e3d(Geo3D g, State3D<R> s, Coef<R> c, Pml3D<R> pm, Step3D<R> a3)
{
    const int i = blockIdx.x * BX + threadIdx.x;
    const int j = blockIdx.y * BY + threadIdx.y;
    const int k = blockIdx.z * BZ + threadIdx.z;
    if (i >= g.n[0] || j >= g.n[1] || k >= g.n[2]) return;
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

}  // namespace

template <typename R>
int launch_step3d(int mode, const Geo3D &g, const State3D<R> &s, const Coef<R> &c, const Pml3D<R> &pm,
                  const Step3D<R> &a, cudaStream_t st)
{
    dim3 block(BX, BY, BZ), grid((g.n[0] + BX - 1) / BX, (g.n[1] + BY - 1) / BY, (g.n[2] + BZ - 1) / BZ);
    k_h3d<R><<<grid, block, 0, st>>>(g, s, c, pm);
    if (mode == 0) k_e3d<R, 0><<<grid, block, 0, st>>>(g, s, c, pm, a);
    else k_e3d<R, 1><<<grid, block, 0, st>>>(g, s, c, pm, a);
    return 2;
}

template int launch_step3d<float>(int, const Geo3D &, const State3D<float> &, const Coef<float> &,
                                  const Pml3D<float> &, const Step3D<float> &, cudaStream_t);
template int launch_step3d<double>(int, const Geo3D &, const State3D<double> &, const Coef<double> &,
                                   const Pml3D<double> &, const Step3D<double> &, cudaStream_t);

}  // namespace fdtd
