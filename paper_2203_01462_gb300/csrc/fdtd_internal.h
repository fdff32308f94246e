// Internal declarations shared by the host orchestration (fdtd_host.cu) and
// the kernel translation units.  Nothing here crosses the C ABI.
#pragma once

#include <vector>

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace fdtd {

// Device error word bits (reported by fdtd_sync).
enum : unsigned { ERR_RANGE = 1u, ERR_NONFINITE = 2u, ERR_UNSTABLE = 4u, ERR_TIMEOUT = 8u };

// Geometry of a 2D TM_z grid: Ez, Hx, Hy on nx x ny nodes with row pitch px
// (elements).  Hx[j][i] sits at (i, j + 1/2), Hy[j][i] at (i + 1/2, j).
struct Geo2D {
    int nx, ny, px, npml;
    int dx0, dy0, dnx, dny;   // design box origin and size (nodes)
    int dxa, dp;              // pitched design arrays: column origin (dx0
                              // rounded down to a multiple of 4) and row
                              // pitch (a multiple of 4); node (i, j) of the
                              // box is element (j - dy0) * dp + (i - dxa)
    int gx0, gy0, gnx, gny;   // gap box
    int sx0, sx1, sy0, sy1;   // source box
};

// Field arrays of one 2D solver state.  J covers the design box only
// (pitched layout, see Geo2D).  CPML convolution terms live in border slabs:
// x-slabs [ny][2 npml] for Ez and Hy, y-slabs [2 npml][px] for Ez and Hx.
template <typename R>
struct State2D {
    R *Ez, *Hx, *Hy, *J;
    R *pezx, *phyx, *pezy, *phxy;
};

// CPML tables along one axis, per node position (E) and half position (H):
// b, c of the recursive convolution and 1 / kappa.
template <typename R>
struct Pml1D {
    const R *bE, *cE, *kiE, *bH, *cH, *kiH;
};

// Step-invariant update coefficients in scaled units: E as is, H~ = eta0 H,
// J~ = J dt / eps0, psi~ = omega_p^2 dt^2, sigma~ = sigma dt / eps0,
// gamma~ = gamma dt.
template <typename R>
struct Coef {
    R S;            // Courant number c0 dt / dx
    R eps_s, eps_g, inv_eps_s, inv_eps_g;
    R eps_sub;      // 3D: background below the substrate plane
    R d_eps;        // eps_inf - eps_s
    R psi, psi_s;   // scaled psi of the metal and of the background
    R sig_max;      // scaled sigma_max, times 4 for the peak-normalised form
    R kJ;           // (1 - gamma~/2) / (1 + gamma~/2)
    R inv1g;        // 1 / (1 + gamma~/2)
    R half1pkJ;     // (1 + kJ) / 2
    // Factors of the three Eq. (25) terms in the adjoint's accumulator, each
    // with its chain-rule factor: d_eps, sig_max and psi - psi_s for a term
    // that is selected (fdtd_set_sensitivity_terms), 0 for one that is not.
    R t_eps, t_sig, t_dpsi;
};

// Constant-memory coefficient slots (one per live context; coef_slots.cuh).
constexpr int COEF_SLOTS = 128;
// Write the coefficients of a slot for the step kernels of one translation
// unit (stream ordered; the host struct may go out of scope on return).
template <typename R>
cudaError_t upload_coef_2d(int slot, const Coef<R> &c, cudaStream_t st);
template <typename R>
cudaError_t upload_coef_3d(int slot, const Coef<R> &c, cudaStream_t st);
template <typename R>
cudaError_t upload_coef_p(int slot, const Coef<R> &c, cudaStream_t st);

// Per-step arguments of the fused step kernel (kernels_2d.cu); the host
// resolves every per-step offset into a base pointer.
template <typename R>
struct Step2D {
    const R *rho_t;      // filtered density on the design box
    const R *src;        // forward: source table entry of this step
    const R *gap_src;    // adjoint: forward gap field E^m (row m of the history)
    R *gap_rec;          // forward: gap-history row receiving E^{n+1} (or null)
    R *rec;              // forward: design-box slot receiving E^{n+1} (or null);
                         // adjoint: design-box forward E^m
    double *G;           // adjoint: sensitivity accumulator
};

// One fused time step of the whole grid, reading state `in`, writing `out`.
// mode 0: forward / recompute; 1: adjoint.
template <typename R>
int launch_step2d(int mode, const Geo2D &g, const State2D<R> &in, const State2D<R> &out, int coef_slot,
                  const Pml1D<R> &px, const Pml1D<R> &py, const Step2D<R> &a, cudaStream_t st, const cudaAccessPolicyWindow *win);

// Blocks of one 2D step launch, and how many of them take the vector path.
void step2d_block_counts(const Geo2D &g, long long *total, long long *vector);

// Auxiliary kernels (kernels_aux.cu).
template <typename R>
void launch_guard(const R *state, long long n, double bound, unsigned *err, unsigned *host_flag, unsigned tag,
                  cudaStream_t st);
template <typename R>
void launch_copy_check_rho(const R *src, R *dst, long long n, unsigned *err, cudaStream_t st);
template <typename T>
void launch_filter_rows(const T *in, T *out, int w, int h, int R_, const T *wts, const T *inv_norm,
                        int transpose, cudaStream_t st);
template <typename T>
void launch_filter_cols(const T *in, T *out, int w, int h, int R_, const T *wts, const T *inv_norm,
                        int transpose, cudaStream_t st);
template <typename R>
void launch_objective(const R *gap_hist, long long count, double coef, double *W, double *W_user, double *part,
                      unsigned *err, cudaStream_t st);
// Blocks of the objective reduction; `part` holds OBJ_BLOCKS doubles.
constexpr int OBJ_BLOCKS = 152 * 8;
// ------------------------------------------------------------------ 3D

// Geometry of a 3D Yee grid of n[0] x n[1] x n[2] nodes; rows padded to px
// nodes, planes of PP = px * n[1] nodes.  Boxes are half-open node ranges.
// Design-box arrays are pitched: dn[2] x dn[1] rows of dp elements starting
// at column dxa; Mdi = dn[2] * dn[1] * dp elements per component.
struct Geo3D {
    int n[3];
    int px;
    long long PP;
    int npml;
    int d0[3], dn[3], dxa, dp;
    long long Mdi;
    int g0[3], gn[3];
    int Mg;
    int s0[3], s1[3], src_comp;
    int sub_hi;
    // plane wave by total-field / scattered-field injection (tfsf = 1): the
    // closed total-field box of positions [tf_lo, tf_hi] (node units)
    int tfsf, tf_lo[3], tf_hi[3];
    int kappa1;  // every CPML kappa is 1 (pml_kappa_max = 1): the 1/kappa tables are all ones
};

// Incident-table row of one step of the plane wave: E_x^n at k = tf_lo[2] ..
// tf_hi[2], then H_y^{n+1/2} at k = tf_lo[2]-1 .. tf_hi[2].
inline int tfsf_row(const Geo3D &g) { return 2 * (g.tf_hi[2] - g.tf_lo[2] + 1) + 1; }

// One 3D solver state: three E, H and J components (J over the pitched
// design box), and the CPML terms of component c for its two derivative
// axes (c+1, c+2 cyclic), each stored in the slabs of that axis.
template <typename R>
struct State3D {
    R *E[3], *H[3], *J[3];
    R *pe[3][2], *ph[3][2];
};

template <typename R>
struct Pml3D {
    const R *bE[3], *cE[3], *kiE[3], *bH[3], *cH[3], *kiH[3];
};

template <typename R>
struct Step3D {
    const R *rho_t;
    const R *src;        // forward: source table entry of this step
    const R *gap_src;    // adjoint: gap rows E^m, [component][M_g]
    R *gap_rec;          // forward: gap rows receiving E^{n+1} (or null)
    R *rec;              // forward: design record slot [component][Mdi] (or null);
                         // adjoint: forward E^m, same layout
    double *G;           // adjoint: sensitivity accumulator [Mdi]
    const R *tf_inc;     // forward with tfsf: incident-table row of this step
};

// 2D with E in plane (the paper's 2D "TM" case): Ex(i, j) on the edge
// (i+1/2, j), Ey(i, j) on (i, j+1/2), Hz(i, j) at (i+1/2, j+1/2); [ny][px]
// arrays.  Design variables, Drude currents and the gap live on edges: for
// component c (0 = x, 1 = y) the edges of the design box form a rectangle
// of array indices with origin d0[c] and extent dn[c] (E_x: dnx x (dny+1),
// E_y: (dnx+1) x dny); their arrays use the pitched layout of the 2D design
// box (column origin dxa[c], pitch dp[c]).
struct GeoP {
    int nx, ny, px, npml;
    int d0[2][2], dn[2][2], dxa[2], dp[2];
    long long Mdi[2];
    int g0[2][2], gn[2][2], Mgc[2];  // gap edges per component; a gap record is Mgc[0] E_x then Mgc[1] E_y values
    int s0[2], s1[2];                // source E_x edges: i in [s0x, s1x), j in [s0y, s1y)
};

// State: fields, per-component Drude currents (pitched design layout) and
// the CPML terms: pexy (Ex, d/dy) and phzy (Hz, d/dy) in the y-slabs,
// [2 npml][px]; peyx (Ey, d/dx) and phzx (Hz, d/dx) in the x-slabs,
// [ny][2 npml].
template <typename R>
struct StateP {
    R *Ex, *Ey, *Hz, *J[2];
    R *pexy, *peyx, *phzx, *phzy;
};

template <typename R>
struct PmlP {
    const R *bE[2], *cE[2], *kiE[2], *bH[2], *cH[2], *kiH[2];  // per axis (0 = x, 1 = y)
};

template <typename R>
struct StepP {
    const R *rho_t[2];   // pitched densities of the E_x and E_y design edges
    const R *src;        // forward: source table entry of this step
    const R *gap_src;    // adjoint: forward gap record E^m
    R *gap_rec;          // forward: gap record receiving E^{n+1} (or null)
    R *rec[2];           // forward: design-edge record slots (or null); adjoint: forward E^m
    double *G[2];        // adjoint: sensitivity accumulators
};

// H then E half steps of the in-plane 2D grid, in place (two launches).
template <typename R>
int launch_stepp(int mode, const GeoP &g, const StateP<R> &s, int coef_slot, const PmlP<R> &pm,
                 const StepP<R> &a, cudaStream_t st);

// Per-step pointers of a run of `count` in-plane steps in one launch.  Mode
// 0 (forward / recompute): step n = n0 + t takes src[n], writes gap row n+1
// of gap (if not null) and the design record slot n - rec0 of rec (if not
// null).  Mode 1 (adjoint): step t takes m = n0 - t, the gap row m as its
// source and the forward fields of slot m - 1 - rec0.
template <typename R>
struct PlanP {
    const R *src;
    R *gap, *rec;
    long long rec_step, Mdi0;   // elements per record slot; offset of the E_y part
    int Mg, rec0, n0, count;
};

// Words of the multi-step launch's barrier (two); whether
// its blocks (one per SM) can all be resident at once on the current device
// (required: they wait on one another).
int stepp_multi_tiles(const GeoP &g);
template <typename R>
bool stepp_multi_fits(const GeoP &g);

// plan.count steps in one cooperative launch (kernels_2dp.cu).  flags: the
// grid barrier's arrival count and generation (count zero between launches);
// a wait longer than `limit` clock cycles sets ERR_TIMEOUT in *err and
// *abort_word.
template <typename R>
int launch_stepp_multi(int mode, const GeoP &g, const StateP<R> &s, int coef_slot, const PmlP<R> &pm,
                       const StepP<R> &base, const PlanP<R> &plan, unsigned phase0, unsigned *flags,
                       unsigned *abort_word, unsigned *err, long long limit, cudaStream_t st);

// One bounded wait on words[0] >= 1 (abort word words[1], error word
// words[2]) that nothing satisfies: it records ERR_TIMEOUT after `limit`
// clock cycles.
void launch_wait_selftest(unsigned *words, long long limit, cudaStream_t st);

// H then E half steps of the whole grid, in place (two launches); a forward
// step with a.tf_inc adds the plane wave's face corrections inside them.
// Returns the launch count.
template <typename R>
int launch_step3d(int mode, const Geo3D &g, const State3D<R> &s, int coef_slot, const Pml3D<R> &pm,
                  const Step3D<R> &a, cudaStream_t st);

// Temporally blocked 2D E_z steps (kernels_tb2d.cu): a block owns a square
// tile (`tile` nodes a side, tb2d_tile) and advances count <= TB_MAX steps
// on it and a halo of count nodes in shared memory, reading state `in` and
// writing its tile into `out`.
// Forward: steps n0 .. n0+count-1 (source row n, gap row n+1, design record
// slot n - rec0); adjoint: m = n0 down to n0-count+1 (gap row m, record slot
// m-1-rec0), G the accumulator.
constexpr int TB_MAX = 8;
template <typename R>
struct Tb2D {
    int count, n0, rec0, tile;
    long long Mdi;
    const R *src;
    R *gap;
    R *rec;
    const R *rho_t;
    double *G;
};
size_t tb2d_smem_bytes(int esz, int T);
// Tile side of the blocked kernel for an nx x ny grid on `sms` SMs.
int tb2d_tile(int nx, int ny, int sms);
// The most steps per launch whose region fits a block's shared memory (and
// the kernels' shared-memory limit raised to it), or 0.
template <typename R>
int tb2d_max_steps();
template <typename R>
int launch_tb2d(int mode, const Geo2D &g, const State2D<R> &in, const State2D<R> &out, int coef_slot,
                const Pml1D<R> &px, const Pml1D<R> &py, const Tb2D<R> &w, cudaStream_t st);
template <typename R>
cudaError_t upload_coef_tb2d(int slot, const Coef<R> &c, cudaStream_t st);

// Several 3D steps in one persistent launch (kernels_3d.cu, k_wave3d).
// The grid is cut into z slabs of two planes; an item is up to `tpi`
// x-adjacent node tiles of one row of one slab, and a job is every item of
// one half step ("phase": 2t = H of step t, 2t+1 = E of step t) on one slab.
// jobs[] lists the 2 count nslab jobs (phase << 16 | slab) in an order in
// which every job comes after the jobs it depends on (E_t(s) on H_t(s),
// H_t(s-1); H_t(s) on E_{t-1}(s), E_{t-1}(s+1)); blocks take the items in
// that order, round-robin, and wait (bounded) on per-slab counters of
// finished items.
template <typename R>
struct Wave3D {
    const int *jobs;
    unsigned *cnt;  // [nslab] H items done, [nslab] E items done, abort word, finished blocks
    int count, nslab, gx, ipr, ips, tpi;
    int n0, rec0;   // forward: steps n0 .. n0+count-1, design record slot n - rec0;
                    // adjoint: m = n0 down to n0-count+1, record slot m-1-rec0
    const R *src;   // forward source table (indexed by n)
    R *gap;         // gap history (forward writes row n+1, adjoint reads row m) or null
    R *rec;         // design records or null (forward)
    const R *tf;    // incident table of the plane wave (forward) or null
    int tf_row;
};

// Job order of one wavefront launch: job (p, s) has key s + lag p and the
// jobs are sorted by key, phase ascending within a key.  lag >= 2.
std::vector<int> wave3d_jobs(int nslab, int count, int lag);
// Blocks one wavefront launch keeps resident (mode 0 forward, 1 adjoint),
// or 0 when the device cannot run it as a cooperative launch.
template <typename R>
int wave3d_blocks(int mode);
// One wavefront launch of w.count steps on `blocks` blocks (cooperative).
// a0 carries rho_t and (adjoint) G; the per-step pointers come from w.
// A wait longer than `limit` clock cycles sets ERR_TIMEOUT in *err and the
// abort word; a launch that finds the abort word set does nothing.
template <typename R>
int launch_wave3d(int mode, const Geo3D &g, const State3D<R> &s, int coef_slot, const Pml3D<R> &pm,
                  const Step3D<R> &a0, const Wave3D<R> &w, int blocks, unsigned *err, long long limit,
                  cudaStream_t st);
constexpr int WAVE3D_TX = 32, WAVE3D_TY = 8, WAVE3D_TZ = 2;  // nodes of one tile

// The incident plane wave of a tfsf grid: one block steps the 1D column
// (E_x, H_y, their z-CPML terms in col, 4 nz words, cleared here) for
// nsteps steps and writes one tfsf_row(g) row per step into tab.  eps_s,
// eps_sub: background permittivities above / below g.sub_hi; S: Courant
// number; src: the source table (scaled current per step).
template <typename R>
void launch_tfsf_column(const Geo3D &g, const Pml3D<R> &pm, R S, R eps_s, R eps_sub, const R *src, int nsteps,
                        R *col, R *tab, cudaStream_t st);

// A forward (recompute) step of one state and an adjoint step of another in
// one launch (independent work; see k_step2d_pair).
template <typename R>
int launch_step2d_pair(const Geo2D &g, const State2D<R> &fin, const State2D<R> &fout, const Step2D<R> &fa,
                       const State2D<R> &ain, const State2D<R> &aout, const Step2D<R> &aa, int coef_slot,
                       const Pml1D<R> &px, const Pml1D<R> &py, cudaStream_t st, const cudaAccessPolicyWindow *win);

// Compact (dnx x dny) <-> pitched (dny rows of dp, box at column off).
template <typename T>
void launch_pitch2d(const T *compact, T *pitched, int dnx, int dny, int off, int dp, cudaStream_t st);
// out (compact) = scale * G (pitched), zero on gap nodes (gap box relative
// to the design box).
void launch_assemble_2d(const double *G, double *out, int dnx, int dny, int off, int dp, int gx0, int gy0,
                        int gnx, int gny, double scale, cudaStream_t st);
void launch_assemble_3d(const double *G, double *out, int dx, int dy, int dz, int off, int dp, int gx0, int gy0,
                        int gz0, int gnx, int gny, int gnz, double scale, cudaStream_t st);
void launch_zero_gap_2d(double *g, int dnx, int gx0, int gy0, int gnx, int gny, cudaStream_t st);
template <typename R>
void launch_to_double(const R *in, double *out, long long n, cudaStream_t st);
template <typename R>
void launch_gap_dft(const R *x, long long nt, int m, double dt, const double *freqs, int nf, double *out,
                    cudaStream_t st);
void launch_copy_bytes(const void *src, void *dst, size_t bytes, cudaStream_t st);

// Optimization-loop kernels (kernels_opt.cu).
template <typename R>
void launch_ascent(R *rho, const double *g, long long n, double move, unsigned long long *gmax, cudaStream_t st);
template <typename R>
void launch_grayness(const R *rt, long long rows, int dnx, int dp, int off, int rows_per_plane, int gx0, int gy0,
                     int gz0, int gnx, int gny, int gnz, double *acc, cudaStream_t st, bool accumulate = false);
void launch_scale1(double *x, double s, cudaStream_t st);
template <typename R>
void launch_threshold(R *rho, long long n, double level, cudaStream_t st);
// The design layout as one or two x-fastest rectangles (w x h x d entries
// from offset off): the node box in TM_z 2D and 3D, the E_x and E_y edge
// rectangles in the in-plane 2D mode.
struct DesignRects {
    int n;
    long long off[2];
    int w[2], h[2], d[2];
};
template <typename T>
void launch_mirror_avg(T *v, const DesignRects &r, int axis, cudaStream_t st);
template <typename T>
void launch_fix(T *rho, double *g, const unsigned char *mask, long long n, double value, cudaStream_t st);

// Block count of the MMA kernels; the context keeps 2 * MMA_BLOCKS doubles of
// per-block partial sums.
constexpr int MMA_BLOCKS = 152 * 8;
template <typename R>
void launch_mma_asymptotes(const R *rho, const double *g, double *state, long long n, int k, double *part,
                           double *sums, cudaStream_t st);
template <typename R>
void launch_mma_solve(const double *state, const double *g, long long n, double s, double raa0, double move, R *out,
                      double *part, double *sums, cudaStream_t st);

// 16-bit checkpoints (kind 1: BF16, 2: FP16) with one float scale per slab
// of SNAP_SLAB consecutive words of the state block.
constexpr long long SNAP_SLAB = 2048;
template <typename R>
void launch_snap_pack(int kind, const R *src, void *dst, float *scales, long long n, cudaStream_t st);
template <typename R>
void launch_snap_unpack(int kind, const void *src, const float *scales, R *dst, long long n, cudaStream_t st);
void launch_zero_bytes(void *dst, size_t bytes, cudaStream_t st);

}  // namespace fdtd

struct fdtd_ctx;
namespace fdtd {
// The gradient of fdtd_gradient with the two filter-transpose intermediates
// taken from `scratch` (two arrays of scratch_per_array doubles of device
// memory) instead of the workspace (fdtd_host.cu).  Only a 2D E_z context
// with a design filter uses them, and only it needs n <= scratch_per_array.
// Returns an fdtd_status value.
int gradient_into(fdtd_ctx *ctx, double *d_grad, size_t n, double *scratch, size_t scratch_per_array);
// The device that was current when the context was created.
int context_device(const fdtd_ctx *ctx);
}  // namespace fdtd
