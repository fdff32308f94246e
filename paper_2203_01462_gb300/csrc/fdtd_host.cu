// Host side of the C ABI declared in include/fdtd.h: configuration checks,
// workspace layout, CPML / source / filter tables, and the time loops of the
// forward run, the checkpointed recompute and the adjoint run.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <memory>
#include <new>
#include <mutex>
#include <vector>

#include "../../include/fdtd.h"
#include "fdtd_internal.h"

using namespace fdtd;

namespace {

constexpr double kC0 = 299792458.0;
constexpr double kMu0 = 1.25663706212e-6;  // CODATA 2018
constexpr double kPi = 3.14159265358979323846;
inline double eps0() { return 1.0 / (kMu0 * kC0 * kC0); }

// Bump allocator over the caller's workspace; a null base only measures.
struct Carver {
    char *base;
    size_t off = 0;
    explicit Carver(void *b) : base((char *)b) {}
    template <typename T>
    T *take(size_t count)
    {
        off = (off + 255) & ~(size_t)255;
        T *p = base ? (T *)(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

bool box_ok(const int *lo, const int *hi, const int *n, int ndim, bool allow_empty)
{
    for (int a = 0; a < 3; ++a) {
        if (a >= ndim) {
            if (lo[a] != 0 || hi[a] != 1) return false;
            continue;
        }
        if (lo[a] < 0 || hi[a] > n[a] || hi[a] < lo[a]) return false;
        if (!allow_empty && hi[a] == lo[a]) return false;
    }
    return true;
}

bool box_inside(const int *lo, const int *hi, const int *olo, const int *ohi, int ndim)
{
    for (int a = 0; a < ndim; ++a)
        if (hi[a] > lo[a] && (lo[a] < olo[a] || hi[a] > ohi[a])) return false;
    return true;
}

long long box_count(const int *lo, const int *hi, int ndim)
{
    long long n = 1;
    for (int a = 0; a < ndim; ++a) n *= (long long)(hi[a] - lo[a]);
    return n;
}

fdtd_status validate(const fdtd_config *c)
{
    if (!c) return FDTD_EINVAL;
    if (c->ndim != 2 && c->ndim != 3) return FDTD_EINVAL;
    if (c->real_bytes != 4 && c->real_bytes != 8) return FDTD_EINVAL;
    if (c->nx < 4 || c->ny < 4 || (c->ndim == 2 ? c->nz != 1 : c->nz < 4)) return FDTD_EINVAL;
    if (c->npml < 0 || c->nx <= 2 * c->npml + 2 || c->ny <= 2 * c->npml + 2 ||
        (c->ndim == 3 && c->nz <= 2 * c->npml + 2))
        return FDTD_EINVAL;
    if (c->ndim == 3 && (c->filter_radius != 0 || c->src_comp < 0 || c->src_comp > 2)) return FDTD_EINVAL;
    if (!(c->dx > 0) || !(c->courant > 0) || c->courant >= 1.0 / sqrt((double)c->ndim)) return FDTD_EINVAL;
    {
        // The Courant limit holds in every medium of the grid: light is
        // 1/sqrt(eps) slower, so S sqrt(d) < sqrt(eps) for the background,
        // the gap, the metal's high-frequency limit eps_inf (design nodes
        // lie between eps_s and eps_inf; the Drude and sigma terms only add
        // to the effective permittivity) and a 3D substrate.
        double emin = std::min(std::min(c->eps_s, c->eps_g), c->eps_inf);
        if (c->ndim == 3 && c->sub_hi > 0) emin = std::min(emin, c->sub_eps);
        if (!(emin > 0) || c->courant * sqrt((double)c->ndim) >= sqrt(emin)) return FDTD_EINVAL;
    }
    if (c->nsteps < 1) return FDTD_EINVAL;
    if (!(c->omega_p > 0) || !(c->psi_s_ratio > 0) || c->gamma_p < 0) return FDTD_EINVAL;
    if (!(c->eps_s > 0) || !(c->eps_g > 0) || !(c->eps_inf > 0)) return FDTD_EINVAL;
    if (c->nbands < 1 || c->nbands > 2) return FDTD_EINVAL;
    if (c->waveform == FDTD_WAVE_GAUSS) {
        if (!(c->tau > 0)) return FDTD_EINVAL;
    } else if (c->waveform == FDTD_WAVE_SINC_HANN) {
        if (!(c->bandwidth > 0) || !isfinite(c->bandwidth) || c->lobes < 1) return FDTD_EINVAL;
    } else {
        return FDTD_EINVAL;
    }
    if (c->pol != FDTD_POL_EZ && c->pol != FDTD_POL_INPLANE) return FDTD_EINVAL;
    if (c->pol == FDTD_POL_INPLANE) {
        // 2D only, no filter; boxes are cell ranges (nx-1 x ny-1 cells); the
        // source box holds E_x edges (i <= nx-2).
        if (c->ndim != 2 || c->filter_radius != 0) return FDTD_EINVAL;
        const int cells[3] = {c->nx - 1, c->ny - 1, 1};
        const int xedges[3] = {c->nx - 1, c->ny, 1};
        if (!box_ok(c->design_lo, c->design_hi, cells, 2, false)) return FDTD_EINVAL;
        if (!box_ok(c->gap_lo, c->gap_hi, cells, 2, true)) return FDTD_EINVAL;
        if (!box_ok(c->src_lo, c->src_hi, xedges, 2, true)) return FDTD_EINVAL;
        if (!box_inside(c->gap_lo, c->gap_hi, c->design_lo, c->design_hi, 2)) return FDTD_EINVAL;
    }
    int n[3] = {c->nx, c->ny, c->nz};
    if (!box_ok(c->design_lo, c->design_hi, n, c->ndim, false)) return FDTD_EINVAL;
    if (!box_ok(c->gap_lo, c->gap_hi, n, c->ndim, true)) return FDTD_EINVAL;
    if (!box_ok(c->src_lo, c->src_hi, n, c->ndim, true)) return FDTD_EINVAL;
    if (!box_inside(c->gap_lo, c->gap_hi, c->design_lo, c->design_hi, c->ndim)) return FDTD_EINVAL;
    if (c->filter_radius < 0 || (c->filter_radius > 0 && !(c->filter_sigma > 0))) return FDTD_EINVAL;
    if (c->snapshot_every < 0) return FDTD_EINVAL;
    if (c->snapshot_dtype < FDTD_SNAP_F32 || c->snapshot_dtype > FDTD_SNAP_F16) return FDTD_EINVAL;
    if (c->accum_kind != FDTD_ACC_F64) return FDTD_EINVAL;
    if (c->sigma_form != FDTD_SIGMA_PAPER && c->sigma_form != FDTD_SIGMA_PEAK_NORMALISED) return FDTD_EINVAL;
    if (c->tfsf != 0 && c->tfsf != 1) return FDTD_EINVAL;
    if (c->tfsf) {
        // x-polarised plane wave along +z: a one-plane source below the
        // total-field box, the box clear of the CPML and strictly around the
        // design box (its corrected faces are background material)
        if (c->ndim != 3 || c->src_comp != 0) return FDTD_EINVAL;
        if (c->src_lo[2] < 1 || c->src_hi[2] != c->src_lo[2] + 1 || c->src_hi[2] > c->tf_lo[2]) return FDTD_EINVAL;
        for (int a = 0; a < 3; ++a) {
            if (c->tf_lo[a] < c->npml + 1 || c->tf_hi[a] > n[a] - c->npml - 2 || c->tf_lo[a] >= c->tf_hi[a])
                return FDTD_EINVAL;
            if (c->tf_lo[a] >= c->design_lo[a] || c->tf_hi[a] < c->design_hi[a]) return FDTD_EINVAL;
        }
    }
    // The step kernels index one array with 32-bit integers.
    const long long px = (c->nx + 31) / 32 * 32;
    if (c->ndim == 2 && px * (long long)c->ny >= (1LL << 31)) return FDTD_EINVAL;
    return FDTD_OK;
}

// ---------------------------------------------------------------- tables

// CPML at a position p (cell units) of an axis with n nodes: depth into the
// layer, polynomial sigma and kappa, linear alpha (Roden-Gedney).
struct PmlPoint { double b, c, ki; };

PmlPoint pml_point(const fdtd_config *c, int n, double p)
{
    PmlPoint r{0.0, 0.0, 1.0};
    const double L = c->npml;
    if (c->npml <= 0) return r;
    double d = 0.0;
    if (p < L) d = L - p;
    else if (p > (n - 1) - L) d = p - ((n - 1) - L);
    if (d <= 0.0) return r;
    const double x = d / L, xm = pow(x, c->pml_m);
    const double eta0 = kMu0 * kC0;
    const double sig = c->pml_sigma_factor * (c->pml_m + 1.0) / (eta0 * c->dx) * xm;
    const double kap = 1.0 + (c->pml_kappa_max - 1.0) * xm;
    const double alp = c->pml_alpha_max * (1.0 - x);
    const double dt = c->courant * c->dx / kC0;
    r.b = exp(-(sig / kap + alp) * dt / eps0());
    r.c = sig > 0.0 ? sig / (sig * kap + kap * kap * alp) * (r.b - 1.0) : 0.0;
    r.ki = 1.0 / kap;
    return r;
}

// Excitation g(t) (see FDTD_WAVE_* in the header): carriers times either a
// Gaussian envelope or the paper's Hanning-smoothed, truncated sinc.
double excitation(const fdtd_config *c, double t)
{
    const double u = t - c->t0;
    double s = 0.0;
    for (int b = 0; b < c->nbands; ++b) s += sin(2.0 * kPi * c->f0[b] * u);
    if (c->waveform == FDTD_WAVE_SINC_HANN) {
        const double half = c->lobes / c->bandwidth;  // T: the window's half-length
        if (!(fabs(u) < half)) return 0.0;
        const double a = kPi * c->bandwidth * u;
        const double envelope = (a == 0.0 ? 1.0 : sin(a) / a) * 0.5 * (1.0 + cos(kPi * u / half));
        return envelope * s;
    }
    const double v = u / c->tau;
    return exp(-v * v) * s;
}

}  // namespace

// -------------------------------------------------------------- context

struct fdtd_ctx {
    fdtd_config cfg;
    cudaStream_t stream = nullptr;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    double dt = 0;
    long long Md = 0, Mg = 0, ncells = 0;
    bool has_design = false, fwd_done = false, adj_done = false;
    double sigma_max = 0.0, gamma_scale = 1.0;
    int terms = FDTD_TERM_ALL;  // Eq. (25) terms the adjoint accumulates
    long long launches = 0, cell_updates = 0;
    int coef_slot = -1;  // constant-memory coefficient slot (coef_slots.cuh)
    // CUDA graphs of whole forward / adjoint passes (replayed when enabled):
    // 0 off, 1 on, 2 automatic (grids of at most GRAPH_AUTO_CELLS nodes).
    int graphs = 2;
    struct Captured {
        cudaGraphExec_t exec = nullptr;
        long long launches = 0, cells = 0;
        int curF = 0, curA = 0;
    } cap[2];
    cudaStream_t capture_stream = nullptr;  // private stream the passes are captured on
    bool capturing = false;                 // a pass is being recorded into a graph
    // Stability guard (fdtd_set_stability_guard): every guard_every forward
    // steps a read-only kernel checks the whole state for non-finite words
    // or magnitudes above the bound.  The host loop that enqueues the steps
    // polls a mapped host word the kernel writes and stops enqueuing once it
    // sees this pass's tag (not possible while capturing a graph; the error
    // word still reports the instability).
    // In-plane 2D contexts: time steps per cooperative launch (1, the
    // default: two launches per step).
    int multi_steps = 1;
    int guard_every = 256;
    double guard_bound = 0.0;  // 0: automatic, see guard_limit()
    unsigned guard_tag = 0;
    unsigned *guard_host = nullptr, *guard_host_dev = nullptr;
    bool guarding = false, guard_stop = false;
    virtual ~fdtd_ctx()
    {
        for (auto &c : cap)
            if (c.exec) cudaGraphExecDestroy(c.exec);
        if (capture_stream) cudaStreamDestroy(capture_stream);
        if (guard_host) cudaFreeHost(guard_host);
    }
    void drop_graphs()
    {
        for (auto &c : cap)
            if (c.exec) {
                cudaGraphExecDestroy(c.exec);
                c = Captured{};
            }
    }
    // Bound on |state word|: the set one, else 1e3 x N x the largest field
    // increment the source gives in one step (src_amp S per band).  A
    // passive medium cannot come near it; growth past it is an instability.
    double guard_limit() const
    {
        double b = guard_bound > 0.0 ? guard_bound
                                     : 1e3 * cfg.nsteps * fabs(cfg.src_amp) * cfg.courant * (double)cfg.nbands;
        if (cfg.real_bytes == 4 && !(b < 1e37)) b = 1e37;
        return b;
    }
    // Called by the forward loops after `done` steps of the current pass.
    // Returns true once the pass should stop (instability seen by the host).
    template <typename R>
    bool guard_after(int done, const void *state, size_t state_bytes)
    {
        if (!guarding || guard_every <= 0 || done % guard_every != 0) return guard_stop;
        launch_guard<R>((const R *)state, (long long)(state_bytes / sizeof(R)), guard_limit(), err_dev(),
                        capturing ? nullptr : guard_host_dev, guard_tag, stream);
        ++launches;
        if (!capturing && guard_host && *(volatile unsigned *)guard_host == guard_tag) guard_stop = true;
        return guard_stop;
    }
    virtual fdtd_status carve(Carver &cv) = 0;
    virtual fdtd_status upload_tables() = 0;
    virtual fdtd_status set_design(const void *d_rho) = 0;
    virtual fdtd_status forward(double *d_W) = 0;
    virtual fdtd_status adjoint() = 0;
    virtual fdtd_status gradient(double *d_grad) = 0;
    virtual fdtd_status gap_history(double *d_out) = 0;
    virtual fdtd_status gap_spectrum(const double *d_freqs, int nf, double *d_out) = 0;
    // fdtd_gradient with the filter-transpose intermediates in s1, s2.
    virtual fdtd_status gradient_scratch(double *d_grad, double *s1, double *s2) = 0;
    // True when gradient_scratch uses s1, s2 (the filter-transpose passes).
    virtual bool gradient_uses_scratch() const { return false; }
    int device = -1;  // the device current at fdtd_create
    // Optimization-loop helpers.
    virtual fdtd_status grayness(double *d_zeta) = 0;
    // L2 residency of the ping-pong state (2D E_z contexts; others ignore it).
    virtual fdtd_status set_l2(double) { return FDTD_OK; }
    // New width of the design filter (2D E_z contexts with a filter).
    virtual fdtd_status set_filter_sigma(double) { return FDTD_EINVAL; }
    // Blocks of one step launch and how many take the vector path (2D E_z).
    virtual void block_counts(long long *total, long long *vec) const { *total = *vec = 0; }
    // True when the passes run as few cooperative launches, which are not
    // captured into graphs.
    virtual bool plain_launches() const { return false; }
    // 3D contexts: up to `steps` steps per wavefront launch (0: split half-step
    // launches).  Returns FDTD_EINVAL for other modes.
    virtual fdtd_status set_wavefront(int) { return FDTD_EINVAL; }
    long long n_free = 0;  // design nodes outside the gap
    virtual void *rho_stage() = 0;
    virtual double *grad_stage() = 0;
    virtual double *W_dev() = 0;
    virtual unsigned *err_dev() = 0;
};

namespace {

fdtd_status cuda_ok(cudaError_t e) { return e == cudaSuccess ? FDTD_OK : FDTD_ECUDA; }
#define FDTD_TRY(x)                          \
    do {                                     \
        fdtd_status s__ = (x);               \
        if (s__ != FDTD_OK) return s__;      \
    } while (0)

constexpr long long GRAPH_AUTO_CELLS = 1LL << 20;

bool use_graphs(const fdtd_ctx *c)
{
    if (c->plain_launches()) return false;
    return c->graphs == 1 || (c->graphs == 2 && c->ncells <= GRAPH_AUTO_CELLS);
}

// Run `enqueue` (which only enqueues work on c->stream) directly, or through
// a CUDA graph captured on its first call and replayed afterwards.  The
// graph is valid for the context's lifetime: every pointer is fixed and the
// coefficients come from the context's constant-memory slot.  Capture runs
// on a private non-blocking stream (the caller's stream may be the legacy
// default stream, which cannot be captured); nothing executes during
// capture, and the graph is launched on the caller's stream.  curF / curA
// receive the ping-pong parities the pass leaves behind.
template <typename F>
fdtd_status run_pass(fdtd_ctx *c, int which, int &curF, int &curA, F &&enqueue)
{
    if (!use_graphs(c)) return enqueue();
    fdtd_ctx::Captured &g = c->cap[which];
    if (!g.exec) {
        if (!c->capture_stream)
            FDTD_TRY(cuda_ok(cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking)));
        const long long l0 = c->launches, c0 = c->cell_updates;
        cudaStream_t user = c->stream;
        c->stream = c->capture_stream;
        fdtd_status s = cuda_ok(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        if (s != FDTD_OK) {
            c->stream = user;
            return s;
        }
        c->capturing = true;
        s = enqueue();
        c->capturing = false;
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
        c->stream = user;
        if (s != FDTD_OK || e != cudaSuccess || !graph) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return s != FDTD_OK ? s : FDTD_ECUDA;
        }
        const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            g.exec = nullptr;
            return FDTD_ECUDA;
        }
        g.launches = c->launches - l0;
        g.cells = c->cell_updates - c0;
        g.curF = curF;
        g.curA = curA;
        c->launches = l0;
        c->cell_updates = c0;
    }
    FDTD_TRY(cuda_ok(cudaGraphLaunch(g.exec, c->stream)));
    c->launches += g.launches;
    c->cell_updates += g.cells;
    curF = g.curF;
    curA = g.curA;
    return FDTD_OK;
}


// Bytes of one checkpoint of a state block of `state_bytes` bytes of R
// words: a plain copy, or 16-bit words plus one float scale per slab (each
// part 256-byte aligned).
template <typename R>
size_t snapshot_bytes(int dtype, size_t state_bytes)
{
    if (dtype == FDTD_SNAP_F32) return state_bytes;
    const long long n = (long long)(state_bytes / sizeof(R));
    const size_t words = ((size_t)n * 2 + 255) & ~(size_t)255;
    const size_t scales = ((size_t)((n + SNAP_SLAB - 1) / SNAP_SLAB) * 4 + 255) & ~(size_t)255;
    return words + scales;
}

template <typename R>
void snapshot_save(int dtype, const char *state, size_t state_bytes, char *snap, cudaStream_t st)
{
    if (dtype == FDTD_SNAP_F32) {
        launch_copy_bytes(state, snap, state_bytes, st);
        return;
    }
    const long long n = (long long)(state_bytes / sizeof(R));
    const size_t words = ((size_t)n * 2 + 255) & ~(size_t)255;
    launch_snap_pack<R>(dtype, (const R *)state, snap, (float *)(snap + words), n, st);
}

template <typename R>
void snapshot_load(int dtype, const char *snap, char *state, size_t state_bytes, cudaStream_t st)
{
    if (dtype == FDTD_SNAP_F32) {
        launch_copy_bytes(snap, state, state_bytes, st);
        return;
    }
    const long long n = (long long)(state_bytes / sizeof(R));
    const size_t words = ((size_t)n * 2 + 255) & ~(size_t)255;
    launch_snap_unpack<R>(dtype, snap, (const float *)(snap + words), (R *)state, n, st);
}

// Step-invariant coefficients in the scaled units of Coef.
template <typename R>
Coef<R> make_coef(const fdtd_config &c, double dt, double sigma_max, double gamma_scale, int terms)
{
    Coef<R> k;
    const double g = c.gamma_p * gamma_scale * dt;
    const double kJ = (1.0 - 0.5 * g) / (1.0 + 0.5 * g);
    const double psi = c.omega_p * c.omega_p * dt * dt;
    k.S = (R)c.courant;
    k.eps_s = (R)c.eps_s;
    k.eps_g = (R)c.eps_g;
    k.eps_sub = (R)c.sub_eps;
    k.inv_eps_s = (R)(1.0 / c.eps_s);
    k.inv_eps_g = (R)(1.0 / c.eps_g);
    k.d_eps = (R)(c.eps_inf - c.eps_s);
    k.psi = (R)psi;
    k.psi_s = (R)(c.psi_s_ratio * psi);
    k.sig_max = (R)(sigma_max * dt / eps0() * (c.sigma_form == FDTD_SIGMA_PEAK_NORMALISED ? 4.0 : 1.0));
    k.kJ = (R)kJ;
    k.inv1g = (R)(1.0 / (1.0 + 0.5 * g));
    k.half1pkJ = (R)(0.5 * (1.0 + kJ));
    // formed in R as the kernels formed these factors before the terms could
    // be selected: with all terms the accumulator uses the same constants
    k.t_eps = (terms & FDTD_TERM_EPS) ? k.d_eps : R(0);
    k.t_sig = (terms & FDTD_TERM_SIGMA) ? k.sig_max : R(0);
    k.t_dpsi = (terms & FDTD_TERM_PSI) ? (R)(k.psi - k.psi_s) : R(0);
    return k;
}

// CPML tables of one axis of n nodes: b, c, 1/kappa at node positions, then
// at half positions (6 n values).
template <typename R>
void fill_pml(const fdtd_config &c, int n, R *t)
{
    for (int i = 0; i < n; ++i) {
        PmlPoint e = pml_point(&c, n, i), h = pml_point(&c, n, i + 0.5);
        t[i] = (R)e.b;
        t[n + i] = (R)e.c;
        t[2 * n + i] = (R)e.ki;
        t[3 * n + i] = (R)h.b;
        t[4 * n + i] = (R)h.c;
        t[5 * n + i] = (R)h.ki;
    }
}

// Source samples J_src dt / eps0 at t = (n + 1/2) dt, n = 0 .. N-1.
template <typename R>
std::vector<R> source_table(const fdtd_config &c, double dt)
{
    std::vector<R> v(c.nsteps);
    for (int n = 0; n < c.nsteps; ++n) v[n] = (R)(c.src_amp * c.courant * excitation(&c, (n + 0.5) * dt));
    return v;
}

template <typename R>
struct Ctx2D final : fdtd_ctx {
    Geo2D geo{};
    State2D<R> F[2]{}, A[2]{};  // ping-pong pairs: forward and adjoint
    char *F_base[2] = {nullptr, nullptr}, *A_base[2] = {nullptr, nullptr};
    int curF = 0, curA = 0;
    // Optional L2 residency of the forward ping-pong pair (fdtd_set_l2_residency).
    // The window goes on the forward and recompute launches only: on the
    // adjoint or the paired launches it measured slower.
    cudaAccessPolicyWindow win = {};
    bool l2 = false;
    const cudaAccessPolicyWindow *winF() const { return l2 ? &win : nullptr; }
    void block_counts(long long *total, long long *vec) const override { step2d_block_counts(geo, total, vec); }
    // Give back the persisting set-aside and demote the lines already marked
    // persisting (best effort for the latter).
    fdtd_status release_l2()
    {
        l2 = false;
        const fdtd_status s = cuda_ok(cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, 0));
        if (cudaCtxResetPersistingL2Cache() != cudaSuccess) cudaGetLastError();
        return s;
    }
    ~Ctx2D() override
    {
        if (l2) release_l2();
    }

    fdtd_status set_l2(double fraction) override
    {
        for (auto &g : cap)
            if (g.exec) {
                cudaGraphExecDestroy(g.exec);
                g.exec = nullptr;
            }
        if (!(fraction > 0)) {
            // release the set-aside: reserved but unused L2 slows every other access
            if (l2) FDTD_TRY(release_l2());
            return FDTD_OK;
        }
        int dev = 0, max_persist = 0, max_window = 0;
        FDTD_TRY(cuda_ok(cudaGetDevice(&dev)));
        FDTD_TRY(cuda_ok(cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, dev)));
        FDTD_TRY(cuda_ok(cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, dev)));
        if (max_persist <= 0 || max_window <= 0) return FDTD_EINVAL;
        const double pair = 2.0 * (double)state_bytes;
        const size_t aside = (size_t)std::min((double)max_persist, fraction * pair);
        FDTD_TRY(cuda_ok(cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, aside)));
        const size_t bytes = (size_t)std::min(pair, (double)max_window);
        win.base_ptr = F_base[0];  // F[0] and F[1] are carved back to back
        win.num_bytes = bytes;
        win.hitRatio = (float)std::min(1.0, (double)aside / (double)bytes);
        win.hitProp = cudaAccessPropertyPersisting;
        win.missProp = cudaAccessPropertyStreaming;
        l2 = true;
        return FDTD_OK;
    }
    size_t state_bytes = 0;
    long long Mdi = 0;  // pitched design-box elements (dny x dp)
    // Temporal blocking (kernels_tb2d.cu): with multi_steps > 1 the forward
    // and the full-history adjoint advance up to min(multi_steps, tb_max)
    // steps per launch.
    int tb_max = 0, tb_tile = 32;
    int tb_steps() const { return (multi_steps > 1 && tb_max > 0) ? std::min(multi_steps, tb_max) : 0; }
    // Steps of the next run from step n (forward): at most T, ending on the
    // guard's multiples while the forward is guarded.
    int tb_run(int n, int end, int T) const
    {
        int e = end;
        if (guarding && guard_every > 0) e = std::min(e, (n / guard_every + 1) * guard_every);
        return std::min(T, e - n);
    }
    R *rho = nullptr, *rhof = nullptr, *rho_t = nullptr, *ftmp = nullptr, *rstage = nullptr;
    double *G = nullptr, *gtmp = nullptr, *gtmp2 = nullptr, *gstage = nullptr;
    R *gap_hist = nullptr, *rec = nullptr, *src_tab = nullptr;
    char *snaps = nullptr;
    size_t snap_stride = 0;
    int nsnap = 0;
    R *pml_tab = nullptr;  // x: 6 * nx, then y: 6 * ny
    Pml1D<R> px{}, py{};
    R *fw_R = nullptr, *fnx_R = nullptr, *fny_R = nullptr;
    double *fw_D = nullptr, *fnx_D = nullptr, *fny_D = nullptr;
    double *misc = nullptr;   // [0] W, [1] ascent max, [4 ..] MMA partial sums
    unsigned *err = nullptr;
    void *rho_stage() override { return rstage; }
    double *grad_stage() override { return gstage; }
    double *W_dev() override { return misc; }
    unsigned *err_dev() override { return err; }

    void carve_state(Carver &cv, State2D<R> &s, char *&base)
    {
        const int np = cfg.npml;
        const size_t grid = (size_t)geo.ny * geo.px;
        size_t start = (cv.off + 255) & ~(size_t)255;
        s.Ez = cv.take<R>(grid);
        s.Hx = cv.take<R>(grid);
        s.Hy = cv.take<R>(grid);
        s.J = cv.take<R>((size_t)Mdi);
        s.pezx = cv.take<R>((size_t)geo.ny * 2 * np);
        s.phyx = cv.take<R>((size_t)geo.ny * 2 * np);
        s.pezy = cv.take<R>((size_t)2 * np * geo.px);
        s.phxy = cv.take<R>((size_t)2 * np * geo.px);
        cv.off = (cv.off + 255) & ~(size_t)255;
        base = cv.base ? cv.base + start : nullptr;
        state_bytes = cv.off - start;
    }

    fdtd_status carve(Carver &cv) override
    {
        const fdtd_config &c = cfg;
        geo.nx = c.nx;
        geo.ny = c.ny;
        geo.px = (c.nx + 31) / 32 * 32;
        geo.npml = c.npml;
        geo.dx0 = c.design_lo[0];
        geo.dy0 = c.design_lo[1];
        geo.dnx = c.design_hi[0] - c.design_lo[0];
        geo.dny = c.design_hi[1] - c.design_lo[1];
        geo.dxa = geo.dx0 & ~3;
        geo.dp = (geo.dx0 + geo.dnx - geo.dxa + 3) & ~3;
        Mdi = (long long)geo.dny * geo.dp;
        geo.gx0 = c.gap_lo[0];
        geo.gy0 = c.gap_lo[1];
        geo.gnx = c.gap_hi[0] - c.gap_lo[0];
        geo.gny = c.gap_hi[1] - c.gap_lo[1];
        geo.sx0 = c.src_lo[0];
        geo.sx1 = c.src_hi[0];
        geo.sy0 = c.src_lo[1];
        geo.sy1 = c.src_hi[1];
        const long long N = c.nsteps;
        for (int b = 0; b < 2; ++b) carve_state(cv, F[b], F_base[b]);
        for (int b = 0; b < 2; ++b) carve_state(cv, A[b], A_base[b]);
        rho = cv.take<R>(Md);
        rhof = cv.take<R>(Md);
        rho_t = cv.take<R>(Mdi);
        ftmp = cv.take<R>(Md);
        rstage = cv.take<R>(Md);
        G = cv.take<double>(Mdi);
        gtmp = cv.take<double>(Md);
        gtmp2 = cv.take<double>(Md);
        gstage = cv.take<double>(Md);
        gap_hist = cv.take<R>((size_t)(N + 1) * (Mg ? Mg : 1));
        const long long K = c.snapshot_every;
        // Full history: N slots.  Checkpoints: two segment buffers of K slots
        // (the adjoint of one segment runs beside the recompute of the next).
        rec = cv.take<R>((size_t)(K > 0 ? 2 * std::min<long long>(K, N) : N) * Mdi);
        nsnap = K > 0 ? (int)((N + K - 1) / K) : 0;
        snap_stride = snapshot_bytes<R>(c.snapshot_dtype, state_bytes);
        snaps = cv.take<char>((size_t)nsnap * snap_stride);
        src_tab = cv.take<R>(N);
        pml_tab = cv.take<R>(6 * (size_t)(c.nx + c.ny));
        const int FR = c.filter_radius;
        fw_R = cv.take<R>(2 * FR + 1);
        fnx_R = cv.take<R>(geo.dnx);
        fny_R = cv.take<R>(geo.dny);
        fw_D = cv.take<double>(2 * FR + 1);
        fnx_D = cv.take<double>(geo.dnx);
        fny_D = cv.take<double>(geo.dny);
        misc = cv.take<double>(4 + 2 * MMA_BLOCKS);
        err = cv.take<unsigned>(4);
        if (pml_tab) {
            R *t = pml_tab;
            px = {t, t + c.nx, t + 2 * c.nx, t + 3 * c.nx, t + 4 * c.nx, t + 5 * c.nx};
            t += 6 * c.nx;
            py = {t, t + c.ny, t + 2 * c.ny, t + 3 * c.ny, t + 4 * c.ny, t + 5 * c.ny};
        }
        return FDTD_OK;
    }

    fdtd_status upload_tables() override
    {
        const fdtd_config &c = cfg;
        std::vector<R> tab(6 * (size_t)(c.nx + c.ny));
        fill_pml<R>(c, c.nx, tab.data());
        fill_pml<R>(c, c.ny, tab.data() + 6 * c.nx);
        std::vector<R> src = source_table<R>(c, dt);
        cudaStream_t st = stream;
        FDTD_TRY(cuda_ok(cudaMemcpyAsync(pml_tab, tab.data(), tab.size() * sizeof(R), cudaMemcpyHostToDevice, st)));
        FDTD_TRY(cuda_ok(cudaMemcpyAsync(src_tab, src.data(), src.size() * sizeof(R), cudaMemcpyHostToDevice, st)));
        FDTD_TRY(upload_filter(c.filter_sigma));
        launch_zero_bytes(err, 4 * sizeof(unsigned), st);
        ++launches;
        tb_max = tb2d_max_steps<R>();
        // Default: temporal blocking on FP32 grids of at most one 32 x 32 tile
        // per SM, where the launch-per-step kernels are single partial waves
        // (measured: 316^2, 7.1 -> 3.4 us per forward step with 32 x 32
        // tiles); larger or FP64 grids run faster one launch per step.  The
        // tile side is the smallest whose tiles still fit one wave.
        {
            int dev = 0, sms = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            tb_tile = tb2d_tile(c.nx, c.ny, sms);
            const long long tiles = (long long)((c.nx + tb_tile - 1) / tb_tile) * ((c.ny + tb_tile - 1) / tb_tile);
            if (sizeof(R) == 4 && tb_max > 0 && tiles <= sms) multi_steps = TB_MAX;
        }
        return cuda_ok(cudaStreamSynchronize(st));
    }

    // Weights exp(-k^2 / (2 sigma^2)), |k| <= filter_radius, of the Gaussian
    // design filter (Eq. 26) and the per-row / per-column normalisations of
    // the truncated window at the box edges, in both precisions.
    fdtd_status upload_filter(double sigma)
    {
        const int FR = cfg.filter_radius;
        std::vector<double> w(2 * FR + 1), nx(geo.dnx), ny(geo.dny);
        for (int k = -FR; k <= FR; ++k) w[k + FR] = FR ? exp(-(double)k * k / (2.0 * sigma * sigma)) : 1.0;
        auto norms = [&](std::vector<double> &v, int n) {
            for (int i = 0; i < n; ++i) {
                double s = 0.0;
                for (int k = -FR; k <= FR; ++k)
                    if (i + k >= 0 && i + k < n) s += w[k + FR];
                v[i] = 1.0 / s;
            }
        };
        norms(nx, geo.dnx);
        norms(ny, geo.dny);
        std::vector<R> wR(w.begin(), w.end()), nxR(nx.begin(), nx.end()), nyR(ny.begin(), ny.end());
        cudaStream_t st = stream;
        FDTD_TRY(cuda_ok(cudaMemcpyAsync(fw_R, wR.data(), wR.size() * sizeof(R), cudaMemcpyHostToDevice, st)));
        FDTD_TRY(cuda_ok(cudaMemcpyAsync(fnx_R, nxR.data(), nxR.size() * sizeof(R), cudaMemcpyHostToDevice, st)));
        FDTD_TRY(cuda_ok(cudaMemcpyAsync(fny_R, nyR.data(), nyR.size() * sizeof(R), cudaMemcpyHostToDevice, st)));
        FDTD_TRY(cuda_ok(cudaMemcpyAsync(fw_D, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice, st)));
        FDTD_TRY(cuda_ok(cudaMemcpyAsync(fnx_D, nx.data(), nx.size() * sizeof(double), cudaMemcpyHostToDevice, st)));
        FDTD_TRY(cuda_ok(cudaMemcpyAsync(fny_D, ny.data(), ny.size() * sizeof(double), cudaMemcpyHostToDevice, st)));
        // the host vectors go out of scope: finish the copies first
        return cuda_ok(cudaStreamSynchronize(st));
    }

    fdtd_status set_filter_sigma(double sigma) override
    {
        if (cfg.filter_radius <= 0) return FDTD_EINVAL;
        FDTD_TRY(upload_filter(sigma));
        cfg.filter_sigma = sigma;
        return FDTD_OK;
    }

    Coef<R> coef() const { return make_coef<R>(cfg, dt, sigma_max, gamma_scale, terms); }

    // A pass enqueues its launches (enqueue_*), directly or as a replayed
    // CUDA graph; the coefficients go to the context's constant slot first.
    fdtd_status forward(double *d_W) override
    {
        FDTD_TRY(cuda_ok(upload_coef_2d<R>(coef_slot, coef(), stream)));
        if (tb_steps()) FDTD_TRY(cuda_ok(upload_coef_tb2d<R>(coef_slot, coef(), stream)));
        int keepA = curA;
        FDTD_TRY(run_pass(this, 0, curF, keepA, [&] { return enqueue_forward(); }));
        if (d_W && d_W != misc)
            FDTD_TRY(cuda_ok(cudaMemcpyAsync(d_W, misc, sizeof(double), cudaMemcpyDeviceToDevice, stream)));
        return check_launch();
    }

    fdtd_status adjoint() override
    {
        FDTD_TRY(cuda_ok(upload_coef_2d<R>(coef_slot, coef(), stream)));
        if (tb_steps()) FDTD_TRY(cuda_ok(upload_coef_tb2d<R>(coef_slot, coef(), stream)));
        return run_pass(this, 1, curF, curA, [&] { return enqueue_adjoint(); });
    }

    fdtd_status check_launch() { return cuda_ok(cudaGetLastError()); }

    fdtd_status set_design(const void *d_rho) override
    {
        cudaStream_t st = stream;
        launch_copy_check_rho<R>((const R *)d_rho, rho, Md, err, st);
        ++launches;
        const int FR = cfg.filter_radius;
        if (FR > 0) {
            launch_filter_rows<R>(rho, ftmp, geo.dnx, geo.dny, FR, fw_R, fnx_R, 0, st);
            launch_filter_cols<R>(ftmp, rhof, geo.dnx, geo.dny, FR, fw_R, fny_R, 0, st);
            launch_pitch2d<R>(rhof, rho_t, geo.dnx, geo.dny, geo.dx0 - geo.dxa, geo.dp, st);
            launches += 3;
        } else {
            launch_pitch2d<R>(rho, rho_t, geo.dnx, geo.dny, geo.dx0 - geo.dxa, geo.dp, st);
            ++launches;
        }
        FDTD_TRY(check_launch());
        unsigned h_err = 0;
        FDTD_TRY(cuda_ok(cudaMemcpyAsync(&h_err, err, sizeof(unsigned), cudaMemcpyDeviceToHost, st)));
        FDTD_TRY(cuda_ok(cudaStreamSynchronize(st)));
        if (h_err & ERR_RANGE) {
            launch_zero_bytes(err, sizeof(unsigned), st);
            cudaStreamSynchronize(st);
            return FDTD_ERANGE;
        }
        return FDTD_OK;
    }

    // Advance the forward state from step n0 by count steps.  gap: record
    // E^{n+1} of the gap; rec_base: record design-box E^{n+1} in slot
    // (n - n0) of rec_base (null: no record).
    void advance_forward(int n0, int count, bool gap, R *rec_base)
    {
        Step2D<R> a{};
        a.rho_t = rho_t;
        if (const int T = tb_steps()) {
            for (int n = n0; n < n0 + count;) {
                Tb2D<R> w{};
                w.count = tb_run(n, n0 + count, T);
                w.tile = tb_tile;
                w.n0 = n;
                w.rec0 = n0;
                w.Mdi = Mdi;
                w.src = src_tab;
                w.gap = (gap && Mg) ? gap_hist : nullptr;
                w.rec = rec_base;
                w.rho_t = rho_t;
                launches += launch_tb2d<R>(0, geo, F[curF], F[curF ^ 1], coef_slot, px, py, w, stream);
                curF ^= 1;
                cell_updates += (long long)w.count * ncells;
                n += w.count;
                if (guard_after<R>(n, F_base[curF], state_bytes)) break;
            }
            return;
        }
        for (int n = n0; n < n0 + count; ++n) {
            a.src = src_tab + n;
            a.gap_rec = (gap && Mg) ? gap_hist + (size_t)(n + 1) * Mg : nullptr;
            a.rec = rec_base ? rec_base + (size_t)(n - n0) * Mdi : nullptr;
            launches += launch_step2d<R>(0, geo, F[curF], F[curF ^ 1], coef_slot, px, py, a, stream, winF());
            curF ^= 1;
            cell_updates += ncells;
            if (guard_after<R>(n + 1, F_base[curF], state_bytes)) break;
        }
    }

    // Adjoint steps for m = m_hi down to m_lo + 1 (adjoint step N - m), the
    // forward E^m of the design box in slot (m - 1 - slot0) of base.
    void advance_adjoint_buf(int m_hi, int m_lo, R *base, int slot0)
    {
        Step2D<R> a{};
        a.rho_t = rho_t;
        a.G = G;
        if (const int T = tb_steps()) {
            for (int m = m_hi; m > m_lo;) {
                Tb2D<R> w{};
                w.count = std::min(T, m - m_lo);
                w.tile = tb_tile;
                w.n0 = m;
                w.rec0 = slot0;
                w.Mdi = Mdi;
                w.gap = Mg ? gap_hist : nullptr;
                w.rec = base;
                w.rho_t = rho_t;
                w.G = G;
                launches += launch_tb2d<R>(1, geo, A[curA], A[curA ^ 1], coef_slot, px, py, w, stream);
                curA ^= 1;
                m -= w.count;
            }
            cell_updates += (long long)(m_hi - m_lo) * ncells;
            return;
        }
        for (int m = m_hi; m > m_lo; --m) {
            a.gap_src = Mg ? gap_hist + (size_t)m * Mg : nullptr;
            a.rec = base + (size_t)(m - 1 - slot0) * Mdi;
            launches += launch_step2d<R>(1, geo, A[curA], A[curA ^ 1], coef_slot, px, py, a, stream, nullptr);
            curA ^= 1;
        }
        cell_updates += (long long)(m_hi - m_lo) * ncells;
    }
    void advance_adjoint(int m_hi, int m_lo, int slot0)
    {
        advance_adjoint_buf(m_hi, m_lo, rec, slot0);
    }

    fdtd_status enqueue_forward()
    {
        cudaStream_t st = stream;
        const int N = cfg.nsteps, K = cfg.snapshot_every;
        curF = 0;
        // Both buffers of the pair: padding words are never written by the
        // step kernel, and 16-bit checkpoints scale by the slab maximum.
        launch_zero_bytes(F_base[0], state_bytes, st);
        launch_zero_bytes(F_base[1], state_bytes, st);
        if (Mg) launch_zero_bytes(gap_hist, Mg * sizeof(R), st);
        launches += 3;
        guarding = true;
        if (K <= 0) {
            advance_forward(0, N, true, rec);
        } else {
            for (int s = 0; s < nsnap; ++s) {
                if (guard_stop) break;
                const int n0 = s * K, cnt = std::min(K, N - n0);
                snapshot_save<R>(cfg.snapshot_dtype, F_base[curF], state_bytes, snaps + (size_t)s * snap_stride, st);
                ++launches;
                advance_forward(n0, cnt, true, nullptr);
            }
        }
        guarding = false;
        if (guard_stop) return FDTD_EUNSTABLE;
        const double coefW = 0.5 * cfg.eps_g * dt * pow(cfg.dx, cfg.ndim);
        launch_objective<R>(gap_hist, (long long)(N + 1) * Mg, coefW, misc, nullptr, misc + 4, err, st);
        ++launches;
        return check_launch();
    }

    fdtd_status enqueue_adjoint()
    {
        cudaStream_t st = stream;
        const int N = cfg.nsteps, K = cfg.snapshot_every;
        curA = 0;
        launch_zero_bytes(A_base[0], state_bytes, st);
        launch_zero_bytes(A_base[1], state_bytes, st);
        launch_zero_bytes(G, Mdi * sizeof(double), st);
        launches += 3;
        if (K <= 0) {
            advance_adjoint(N, 0, 0);
            return check_launch();
        }
        // Segments in reverse.  Segment s covers steps [s K, min(s K + K, N));
        // its recomputed design-box fields go to buffer s % 2.  The adjoint
        // steps of segment s run in the same launches as the recompute of
        // segment s - 1 (independent states and buffers).
        auto seg_lo = [&](int s) { return s * K; };
        auto seg_hi = [&](int s) { return std::min(s * K + K, N); };
        auto buf = [&](int s) { return rec + (size_t)(s % 2) * K * Mdi; };
        auto restore = [&](int s) {
            snapshot_load<R>(cfg.snapshot_dtype, snaps + (size_t)s * snap_stride, F_base[curF], state_bytes, st);
            ++launches;
        };
        if (tb_steps()) {
            // temporally blocked: each segment's recompute, then its adjoint
            // (the blocked kernels' results do not depend on how the steps
            // are grouped into launches, so lossless checkpoints reproduce
            // the full-history pass bit for bit)
            for (int s = nsnap - 1; s >= 0; --s) {
                restore(s);
                advance_forward(seg_lo(s), seg_hi(s) - seg_lo(s), false, buf(0));
                advance_adjoint_buf(seg_hi(s), seg_lo(s), buf(0), seg_lo(s));
            }
            return check_launch();
        }
        restore(nsnap - 1);
        advance_forward(seg_lo(nsnap - 1), seg_hi(nsnap - 1) - seg_lo(nsnap - 1), false, buf(nsnap - 1));
        for (int s = nsnap - 1; s >= 1; --s) {
            restore(s - 1);
            const int f0 = seg_lo(s - 1), nf = seg_hi(s - 1) - f0;  // recompute of segment s - 1
            const int a_hi = seg_hi(s), a_lo = seg_lo(s);          // adjoint m = a_hi .. a_lo + 1
            const int pairs = std::min(nf, a_hi - a_lo);
            Step2D<R> fa{}, aa{};
            fa.rho_t = aa.rho_t = rho_t;
            aa.G = G;
            for (int t = 0; t < pairs; ++t) {
                const int n = f0 + t, m = a_hi - t;
                fa.src = src_tab + n;
                fa.rec = buf(s - 1) + (size_t)t * Mdi;
                aa.gap_src = Mg ? gap_hist + (size_t)m * Mg : nullptr;
                aa.rec = buf(s) + (size_t)(m - 1 - a_lo) * Mdi;
                launches += launch_step2d_pair<R>(geo, F[curF], F[curF ^ 1], fa, A[curA], A[curA ^ 1], aa, coef_slot, px,
                                                  py, stream, nullptr);
                curF ^= 1;
                curA ^= 1;
            }
            cell_updates += 2LL * pairs * ncells;
            if (nf > pairs) advance_forward(f0 + pairs, nf - pairs, false, buf(s - 1) + (size_t)pairs * Mdi);
            if (a_hi - a_lo > pairs) advance_adjoint_buf(a_hi - pairs, a_lo, buf(s), a_lo);
        }
        advance_adjoint_buf(seg_hi(0), seg_lo(0), buf(0), seg_lo(0));
        return check_launch();
    }

    fdtd_status gradient(double *d_grad) override
    {
        cudaStream_t st = stream;
        const double scale = dt * pow(cfg.dx, cfg.ndim);
        const int FR = cfg.filter_radius;
        if (FR > 0) {
            launch_assemble_2d(G, gtmp, geo.dnx, geo.dny, geo.dx0 - geo.dxa, geo.dp, geo.gx0 - geo.dx0,
                               geo.gy0 - geo.dy0, geo.gnx, geo.gny, scale, st);
            launch_filter_rows<double>(gtmp, gtmp2, geo.dnx, geo.dny, FR, fw_D, fnx_D, 1, st);
            launch_filter_cols<double>(gtmp2, d_grad, geo.dnx, geo.dny, FR, fw_D, fny_D, 1, st);
            launch_zero_gap_2d(d_grad, geo.dnx, geo.gx0 - geo.dx0, geo.gy0 - geo.dy0, geo.gnx, geo.gny, st);
            launches += 4;
        } else {
            launch_assemble_2d(G, d_grad, geo.dnx, geo.dny, geo.dx0 - geo.dxa, geo.dp, geo.gx0 - geo.dx0,
                               geo.gy0 - geo.dy0, geo.gnx, geo.gny, scale, st);
            ++launches;
        }
        return check_launch();
    }

    fdtd_status grayness(double *d_zeta) override
    {
        launch_grayness<R>(rho_t, geo.dny, geo.dnx, geo.dp, geo.dx0 - geo.dxa, geo.dny, geo.gx0 - geo.dx0,
                           geo.gy0 - geo.dy0, 0, geo.gnx, geo.gny, 1, d_zeta, stream);
        launch_scale1(d_zeta, n_free > 0 ? 4.0 / (double)n_free : 0.0, stream);
        launches += 3;
        return check_launch();
    }

    bool gradient_uses_scratch() const override { return cfg.filter_radius > 0; }
    fdtd_status gradient_scratch(double *d_grad, double *s1, double *s2) override
    {
        cudaStream_t st = stream;
        const double scale = dt * pow(cfg.dx, cfg.ndim);
        const int FR = cfg.filter_radius;
        if (FR > 0) {
            launch_assemble_2d(G, s1, geo.dnx, geo.dny, geo.dx0 - geo.dxa, geo.dp, geo.gx0 - geo.dx0,
                               geo.gy0 - geo.dy0, geo.gnx, geo.gny, scale, st);
            launch_filter_rows<double>(s1, s2, geo.dnx, geo.dny, FR, fw_D, fnx_D, 1, st);
            launch_filter_cols<double>(s2, d_grad, geo.dnx, geo.dny, FR, fw_D, fny_D, 1, st);
            launch_zero_gap_2d(d_grad, geo.dnx, geo.gx0 - geo.dx0, geo.gy0 - geo.dy0, geo.gnx, geo.gny, st);
            launches += 4;
        } else {
            launch_assemble_2d(G, d_grad, geo.dnx, geo.dny, geo.dx0 - geo.dxa, geo.dp, geo.gx0 - geo.dx0,
                               geo.gy0 - geo.dy0, geo.gnx, geo.gny, scale, st);
            ++launches;
        }
        return check_launch();
    }

    fdtd_status gap_history(double *d_out) override
    {
        launch_to_double<R>(gap_hist, d_out, (long long)(cfg.nsteps + 1) * Mg, stream);
        ++launches;
        return check_launch();
    }
    fdtd_status gap_spectrum(const double *d_freqs, int nf, double *d_out) override
    {
        launch_gap_dft<R>(gap_hist, (long long)cfg.nsteps + 1, (int)Mg, dt, d_freqs, nf, d_out, stream);
        ++launches;
        return check_launch();
    }
};

// ------------------------------------------------------ 2D, E in plane

// Edges of a cell box [lo, hi) per component, as array-index rectangles:
// E_x edges i in [lo_x, hi_x), j in [lo_y, hi_y]; E_y edges i in
// [lo_x, hi_x], j in [lo_y, hi_y).
void edge_rect(const int *lo, const int *hi, int cc, int *o, int *n)
{
    const int w = hi[0] - lo[0], h = hi[1] - lo[1];
    o[0] = lo[0];
    o[1] = lo[1];
    if (w <= 0 || h <= 0) {
        n[0] = n[1] = 0;
        return;
    }
    n[0] = cc == 0 ? w : w + 1;
    n[1] = cc == 0 ? h + 1 : h;
}

long long edge_total(const int *lo, const int *hi)
{
    long long t = 0;
    for (int cc = 0; cc < 2; ++cc) {
        int o[2], n[2];
        edge_rect(lo, hi, cc, o, n);
        t += (long long)n[0] * n[1];
    }
    return t;
}

template <typename R>
struct CtxP final : fdtd_ctx {
    GeoP geo{};
    StateP<R> F{}, A{};  // updated in place (split H and E launches)
    char *F_base = nullptr, *A_base = nullptr;
    size_t state_bytes = 0;
    long long Mdx = 0;  // design entries of the E_x edges (first part of rho)
    R *rho = nullptr, *rho_t[2] = {nullptr, nullptr}, *rstage = nullptr;
    double *G[2] = {nullptr, nullptr}, *gstage = nullptr;
    R *gap_hist = nullptr, *rec = nullptr, *src_tab = nullptr;
    char *snaps = nullptr;
    size_t snap_stride = 0;
    int nsnap = 0;
    R *pml_tab = nullptr;
    PmlP<R> pm{};
    double *misc = nullptr;
    unsigned *err = nullptr;
    // Several steps per cooperative launch (k_stepp_multi): the barrier's
    // words (arrival count, generation), then the abort word; the pass's
    // count of half steps so far; whether the launch can be resident.
    unsigned *coop = nullptr;
    int ntiles = 0;
    unsigned coop_phase = 0;
    bool multi_fits = false;
    static constexpr long long WAIT_CYCLES = 2000000000LL;  // about one second

    void *rho_stage() override { return rstage; }
    double *grad_stage() override { return gstage; }
    double *W_dev() override { return misc; }
    unsigned *err_dev() override { return err; }

    long long Mdi_all() const { return geo.Mdi[0] + geo.Mdi[1]; }
    bool multi() const { return multi_fits && multi_steps > 1; }
    bool plain_launches() const override { return multi(); }
    // Steps per launch, a divisor of the guard interval so that a launch
    // ends on every step the guard checks.
    int chunk() const
    {
        int c = multi_steps;
        if (guard_every > 0) {
            int a = c, b = guard_every;
            while (b) {
                const int t = a % b;
                a = b;
                b = t;
            }
            c = a;
        }
        return c > 1 ? c : 1;
    }
    void reset_coop()
    {
        launch_zero_bytes(coop, (size_t)(ntiles + 2) * sizeof(unsigned), stream);
        ++launches;
        coop_phase = 0;
    }
    // Steps [a, b) of one plan (forward: a..b-1; adjoint: m = a down to b+1)
    // in one cooperative launch.
    void launch_multi(int mode, const StateP<R> &st, PlanP<R> plan)
    {
        StepP<R> base = step_args();
        if (mode == 1) {
            base.G[0] = G[0];  // the adjoint's sensitivity accumulators
            base.G[1] = G[1];
        }
        launches += launch_stepp_multi<R>(mode, geo, st, coef_slot, pm, base, plan, coop_phase, coop, coop + ntiles,
                                          err, WAIT_CYCLES, stream);
        coop_phase += 2u * (unsigned)plan.count;
        cell_updates += (long long)plan.count * ncells;
    }

    void carve_state(Carver &cv, StateP<R> &s, char *&base)
    {
        const size_t grid = (size_t)geo.px * geo.ny, np2 = 2 * (size_t)cfg.npml;
        size_t start = (cv.off + 255) & ~(size_t)255;
        s.Ex = cv.take<R>(grid);
        s.Ey = cv.take<R>(grid);
        s.Hz = cv.take<R>(grid);
        s.J[0] = cv.take<R>((size_t)geo.Mdi[0]);
        s.J[1] = cv.take<R>((size_t)geo.Mdi[1]);
        s.pexy = cv.take<R>(np2 * geo.px);
        s.phzy = cv.take<R>(np2 * geo.px);
        s.peyx = cv.take<R>((size_t)geo.ny * np2);
        s.phzx = cv.take<R>((size_t)geo.ny * np2);
        cv.off = (cv.off + 255) & ~(size_t)255;
        base = cv.base ? cv.base + start : nullptr;
        state_bytes = cv.off - start;
    }

    fdtd_status carve(Carver &cv) override
    {
        const fdtd_config &c = cfg;
        geo.nx = c.nx;
        geo.ny = c.ny;
        geo.px = (c.nx + 31) / 32 * 32;
        geo.npml = c.npml;
        for (int cc = 0; cc < 2; ++cc) {
            edge_rect(c.design_lo, c.design_hi, cc, geo.d0[cc], geo.dn[cc]);
            edge_rect(c.gap_lo, c.gap_hi, cc, geo.g0[cc], geo.gn[cc]);
            geo.Mgc[cc] = geo.gn[cc][0] * geo.gn[cc][1];
            geo.dxa[cc] = geo.d0[cc][0] & ~3;
            geo.dp[cc] = (geo.d0[cc][0] + geo.dn[cc][0] - geo.dxa[cc] + 3) & ~3;
            geo.Mdi[cc] = (long long)geo.dn[cc][1] * geo.dp[cc];
        }
        Mdx = (long long)geo.dn[0][0] * geo.dn[0][1];
        for (int a = 0; a < 2; ++a) {
            geo.s0[a] = c.src_lo[a];
            geo.s1[a] = c.src_hi[a];
        }
        const long long N = c.nsteps;
        carve_state(cv, F, F_base);
        carve_state(cv, A, A_base);
        rho = cv.take<R>(Md);
        rho_t[0] = cv.take<R>((size_t)geo.Mdi[0]);
        rho_t[1] = cv.take<R>((size_t)geo.Mdi[1]);
        rstage = cv.take<R>(Md);
        G[0] = cv.take<double>((size_t)geo.Mdi[0]);
        G[1] = cv.take<double>((size_t)geo.Mdi[1]);
        gstage = cv.take<double>(Md);
        gap_hist = cv.take<R>((size_t)(N + 1) * (Mg ? Mg : 1));
        const long long K = c.snapshot_every;
        rec = cv.take<R>((size_t)(K > 0 ? std::min<long long>(K, N) : N) * Mdi_all());
        nsnap = K > 0 ? (int)((N + K - 1) / K) : 0;
        snap_stride = snapshot_bytes<R>(c.snapshot_dtype, state_bytes);
        snaps = cv.take<char>((size_t)nsnap * snap_stride);
        src_tab = cv.take<R>(N);
        pml_tab = cv.take<R>(6 * (size_t)(c.nx + c.ny));
        misc = cv.take<double>(4 + 2 * MMA_BLOCKS);
        err = cv.take<unsigned>(4);
        ntiles = stepp_multi_tiles(geo);
        coop = cv.take<unsigned>((size_t)ntiles + 2);
        if (pml_tab) {
            R *t = pml_tab;
            const int nn[2] = {c.nx, c.ny};
            for (int a = 0; a < 2; ++a) {
                const int n = nn[a];
                pm.bE[a] = t; pm.cE[a] = t + n; pm.kiE[a] = t + 2 * n;
                pm.bH[a] = t + 3 * n; pm.cH[a] = t + 4 * n; pm.kiH[a] = t + 5 * n;
                t += 6 * n;
            }
        }
        return FDTD_OK;
    }

    fdtd_status upload_tables() override
    {
        const fdtd_config &c = cfg;
        std::vector<R> tab(6 * (size_t)(c.nx + c.ny));
        fill_pml<R>(c, c.nx, tab.data());
        fill_pml<R>(c, c.ny, tab.data() + 6 * c.nx);
        std::vector<R> src = source_table<R>(c, dt);
        cudaStream_t st = stream;
        FDTD_TRY(cuda_ok(cudaMemcpyAsync(pml_tab, tab.data(), tab.size() * sizeof(R), cudaMemcpyHostToDevice, st)));
        FDTD_TRY(cuda_ok(cudaMemcpyAsync(src_tab, src.data(), src.size() * sizeof(R), cudaMemcpyHostToDevice, st)));
        launch_zero_bytes(err, 4 * sizeof(unsigned), st);
        ++launches;
        multi_fits = stepp_multi_fits<R>(geo);
        return cuda_ok(cudaStreamSynchronize(st));
    }

    Coef<R> coef() const { return make_coef<R>(cfg, dt, sigma_max, gamma_scale, terms); }

    fdtd_status forward(double *d_W) override
    {
        FDTD_TRY(cuda_ok(upload_coef_p<R>(coef_slot, coef(), stream)));
        int f = 0, a = 0;
        FDTD_TRY(run_pass(this, 0, f, a, [&] { return enqueue_forward(); }));
        if (d_W && d_W != misc)
            FDTD_TRY(cuda_ok(cudaMemcpyAsync(d_W, misc, sizeof(double), cudaMemcpyDeviceToDevice, stream)));
        return check_launch();
    }

    fdtd_status adjoint() override
    {
        FDTD_TRY(cuda_ok(upload_coef_p<R>(coef_slot, coef(), stream)));
        int f = 0, a = 0;
        return run_pass(this, 1, f, a, [&] { return enqueue_adjoint(); });
    }
    fdtd_status check_launch() { return cuda_ok(cudaGetLastError()); }

    fdtd_status set_design(const void *d_rho) override
    {
        cudaStream_t st = stream;
        launch_copy_check_rho<R>((const R *)d_rho, rho, Md, err, st);
        launch_pitch2d<R>(rho, rho_t[0], geo.dn[0][0], geo.dn[0][1], geo.d0[0][0] - geo.dxa[0], geo.dp[0], st);
        launch_pitch2d<R>(rho + Mdx, rho_t[1], geo.dn[1][0], geo.dn[1][1], geo.d0[1][0] - geo.dxa[1], geo.dp[1], st);
        launches += 3;
        FDTD_TRY(check_launch());
        unsigned h_err = 0;
        FDTD_TRY(cuda_ok(cudaMemcpyAsync(&h_err, err, sizeof(unsigned), cudaMemcpyDeviceToHost, st)));
        FDTD_TRY(cuda_ok(cudaStreamSynchronize(st)));
        if (h_err & ERR_RANGE) {
            launch_zero_bytes(err, sizeof(unsigned), st);
            cudaStreamSynchronize(st);
            return FDTD_ERANGE;
        }
        return FDTD_OK;
    }

    StepP<R> step_args() const
    {
        StepP<R> a{};
        a.rho_t[0] = rho_t[0];
        a.rho_t[1] = rho_t[1];
        return a;
    }

    void advance_forward(int n0, int count, bool gap, R *rec_base)
    {
        if (multi()) {
            // runs of steps that end on multiples of chunk(), which divides
            // the guard interval, so the guard sees every step it checks
            const int cs = chunk();
            for (int n = n0; n < n0 + count;) {
                const int n1 = std::min(n0 + count, (n / cs + 1) * cs);
                PlanP<R> pl{};
                pl.src = src_tab;
                pl.gap = (gap && Mg) ? gap_hist : nullptr;
                pl.rec = rec_base;
                pl.rec_step = Mdi_all();
                pl.Mdi0 = geo.Mdi[0];
                pl.Mg = (int)Mg;
                pl.rec0 = n0;
                pl.n0 = n;
                pl.count = n1 - n;
                launch_multi(0, F, pl);
                n = n1;
                if (guard_after<R>(n, F_base, state_bytes)) break;
            }
            return;
        }
        StepP<R> a = step_args();
        for (int n = n0; n < n0 + count; ++n) {
            a.src = src_tab + n;
            a.gap_rec = (gap && Mg) ? gap_hist + (size_t)(n + 1) * Mg : nullptr;
            R *slot = rec_base ? rec_base + (size_t)(n - n0) * Mdi_all() : nullptr;
            a.rec[0] = slot;
            a.rec[1] = slot ? slot + geo.Mdi[0] : nullptr;
            launches += launch_stepp<R>(0, geo, F, coef_slot, pm, a, stream);
            cell_updates += ncells;
            if (guard_after<R>(n + 1, F_base, state_bytes)) break;
        }
    }

    void advance_adjoint(int m_hi, int m_lo, int slot0)
    {
        if (multi()) {
            for (int m = m_hi; m > m_lo;) {
                const int cnt = std::min(multi_steps, m - m_lo);
                PlanP<R> pl{};
                pl.gap = Mg ? gap_hist : nullptr;
                pl.rec = rec;
                pl.rec_step = Mdi_all();
                pl.Mdi0 = geo.Mdi[0];
                pl.Mg = (int)Mg;
                pl.rec0 = slot0;
                pl.n0 = m;
                pl.count = cnt;
                launch_multi(1, A, pl);
                m -= cnt;
            }
            return;
        }
        StepP<R> a = step_args();
        a.G[0] = G[0];
        a.G[1] = G[1];
        for (int m = m_hi; m > m_lo; --m) {
            a.gap_src = Mg ? gap_hist + (size_t)m * Mg : nullptr;
            R *slot = rec + (size_t)(m - 1 - slot0) * Mdi_all();
            a.rec[0] = slot;
            a.rec[1] = slot + geo.Mdi[0];
            launches += launch_stepp<R>(1, geo, A, coef_slot, pm, a, stream);
        }
        cell_updates += (long long)(m_hi - m_lo) * ncells;
    }

    fdtd_status enqueue_forward()
    {
        cudaStream_t st = stream;
        const int N = cfg.nsteps, K = cfg.snapshot_every;
        launch_zero_bytes(F_base, state_bytes, st);
        if (Mg) launch_zero_bytes(gap_hist, Mg * sizeof(R), st);
        launches += 2;
        if (multi()) reset_coop();
        guarding = true;
        if (K <= 0) {
            advance_forward(0, N, true, rec);
        } else {
            for (int s = 0; s < nsnap; ++s) {
                if (guard_stop) break;
                const int n0 = s * K, cnt = std::min(K, N - n0);
                snapshot_save<R>(cfg.snapshot_dtype, F_base, state_bytes, snaps + (size_t)s * snap_stride, st);
                ++launches;
                advance_forward(n0, cnt, true, nullptr);
            }
        }
        guarding = false;
        if (guard_stop) return FDTD_EUNSTABLE;
        const double coefW = 0.5 * cfg.eps_g * dt * cfg.dx * cfg.dx;
        launch_objective<R>(gap_hist, (long long)(N + 1) * Mg, coefW, misc, nullptr, misc + 4, err, st);
        ++launches;
        return check_launch();
    }

    fdtd_status enqueue_adjoint()
    {
        cudaStream_t st = stream;
        const int N = cfg.nsteps, K = cfg.snapshot_every;
        launch_zero_bytes(A_base, state_bytes, st);
        launch_zero_bytes(G[0], geo.Mdi[0] * sizeof(double), st);
        launch_zero_bytes(G[1], geo.Mdi[1] * sizeof(double), st);
        launches += 3;
        if (multi()) reset_coop();
        if (K <= 0) {
            advance_adjoint(N, 0, 0);
        } else {
            for (int s = nsnap - 1; s >= 0; --s) {
                const int n0 = s * K, n1 = std::min(n0 + K, N);
                snapshot_load<R>(cfg.snapshot_dtype, snaps + (size_t)s * snap_stride, F_base, state_bytes, st);
                ++launches;
                advance_forward(n0, n1 - n0, false, rec);
                advance_adjoint(n1, n0, n0);
            }
        }
        return check_launch();
    }

    fdtd_status gradient(double *d_grad) override
    {
        const double scale = dt * cfg.dx * cfg.dx;
        for (int cc = 0; cc < 2; ++cc)
            launch_assemble_2d(G[cc], d_grad + (cc ? Mdx : 0), geo.dn[cc][0], geo.dn[cc][1],
                               geo.d0[cc][0] - geo.dxa[cc], geo.dp[cc], geo.g0[cc][0] - geo.d0[cc][0],
                               geo.g0[cc][1] - geo.d0[cc][1], geo.gn[cc][0], geo.gn[cc][1], scale, stream);
        launches += 2;
        return check_launch();
    }

    fdtd_status grayness(double *d_zeta) override
    {
        for (int cc = 0; cc < 2; ++cc)
            launch_grayness<R>(rho_t[cc], geo.dn[cc][1], geo.dn[cc][0], geo.dp[cc], geo.d0[cc][0] - geo.dxa[cc],
                               geo.dn[cc][1], geo.g0[cc][0] - geo.d0[cc][0], geo.g0[cc][1] - geo.d0[cc][1], 0,
                               geo.gn[cc][0], geo.gn[cc][1], 1, d_zeta, stream, cc == 1);
        launch_scale1(d_zeta, n_free > 0 ? 4.0 / (double)n_free : 0.0, stream);
        launches += 4;
        return check_launch();
    }

    fdtd_status gradient_scratch(double *d_grad, double *, double *) override { return gradient(d_grad); }

    fdtd_status gap_history(double *d_out) override
    {
        launch_to_double<R>(gap_hist, d_out, (long long)(cfg.nsteps + 1) * Mg, stream);
        ++launches;
        return check_launch();
    }
    fdtd_status gap_spectrum(const double *d_freqs, int nf, double *d_out) override
    {
        launch_gap_dft<R>(gap_hist, (long long)cfg.nsteps + 1, (int)Mg, dt, d_freqs, nf, d_out, stream);
        ++launches;
        return check_launch();
    }
};

// ------------------------------------------------------------------ 3D

template <typename R>
struct Ctx3D final : fdtd_ctx {
    Geo3D geo{};
    State3D<R> F{}, A{};  // updated in place (split H and E launches)
    char *F_base = nullptr, *A_base = nullptr;
    size_t state_bytes = 0;
    long long Mdi = 0;
    R *rho = nullptr, *rho_t = nullptr, *rstage = nullptr;
    double *G = nullptr, *gstage = nullptr;
    R *gap_hist = nullptr, *rec = nullptr, *src_tab = nullptr;
    char *snaps = nullptr;
    size_t snap_stride = 0;
    int nsnap = 0;
    R *pml_tab = nullptr;
    Pml3D<R> pm{};
    double *misc = nullptr;
    unsigned *err = nullptr;
    R *tf_tab = nullptr, *tf_col = nullptr;  // plane wave: incident table, column state

    // Wavefront launches (k_wave3d): per-slab counters and the job lists of
    // launches of 1 .. WAVE_MAX steps.
    static constexpr int WAVE_MAX = 8;
    static constexpr long long WAIT_CYCLES = 2000000000LL;  // about one second
    unsigned *wcnt = nullptr;
    int *wjobs = nullptr;
    int nslab = 0, wgx = 0, wtpi = 1, wipr = 0, wips = 0;
    int wave_req = 0;                    // requested steps per launch (0: half-step launches)
    int wave_blocks[2] = {0, 0};         // resident blocks (forward, adjoint kernel); 0: unavailable
    int wave_lag[WAVE_MAX + 1] = {};
    long long wave_off[WAVE_MAX + 1] = {};
    double l2_budget = 0.0;

    bool wave_on() const { return wave_req > 0 && wave_blocks[0] > 0 && wave_blocks[1] > 0; }
    bool plain_launches() const override { return wave_on(); }
    fdtd_status set_wavefront(int steps) override
    {
        if (steps < 0 || steps > WAVE_MAX) return FDTD_EINVAL;
        if (steps > 0 && (wave_blocks[0] <= 0 || wave_blocks[1] <= 0)) return FDTD_ECUDA;
        wave_req = steps;
        return FDTD_OK;
    }
    // Steps per launch: the largest count up to the request whose L2 window
    // (the slabs between the leading H and the trailing E job, lag (2c - 1)
    // + 2 slabs of E and H) fits the budget.
    int wave_count() const
    {
        const double slab = 2.0 * (double)geo.PP * 6.0 * sizeof(R);
        int best = 1;
        for (int c = 2; c <= wave_req; ++c)
            if ((wave_lag[c] * (2.0 * c - 1.0) + 2.0) * slab <= l2_budget) best = c;
        return best;
    }
    Wave3D<R> wave_plan(int count) const
    {
        Wave3D<R> w{};
        w.jobs = wjobs + wave_off[count];
        w.cnt = wcnt;
        w.count = count;
        w.nslab = nslab;
        w.gx = wgx;
        w.ipr = wipr;
        w.ips = wips;
        w.tpi = wtpi;
        w.tf_row = tf_tab ? tfsf_row(geo) : 0;
        return w;
    }
    void wave_reset()
    {
        launch_zero_bytes(wcnt, (size_t)(2 * nslab + 2) * sizeof(unsigned), stream);
        ++launches;
    }

    void *rho_stage() override { return rstage; }
    double *grad_stage() override { return gstage; }
    double *W_dev() override { return misc; }
    unsigned *err_dev() override { return err; }

    size_t slab_elems(int ax) const
    {
        const int np2 = 2 * cfg.npml;
        if (ax == 0) return (size_t)geo.n[2] * geo.n[1] * np2;
        if (ax == 1) return (size_t)geo.n[2] * np2 * geo.px;
        return (size_t)np2 * geo.n[1] * geo.px;
    }

    void carve_state(Carver &cv, State3D<R> &s, char *&base)
    {
        const size_t grid = (size_t)geo.PP * geo.n[2];
        size_t start = (cv.off + 255) & ~(size_t)255;
        for (int c = 0; c < 3; ++c) s.E[c] = cv.take<R>(grid);
        for (int c = 0; c < 3; ++c) s.H[c] = cv.take<R>(grid);
        for (int c = 0; c < 3; ++c) s.J[c] = cv.take<R>((size_t)Mdi);
        for (int c = 0; c < 3; ++c)
            for (int t = 0; t < 2; ++t) {
                const int ax = (c + 1 + t) % 3;
                s.pe[c][t] = cv.take<R>(slab_elems(ax));
                s.ph[c][t] = cv.take<R>(slab_elems(ax));
            }
        cv.off = (cv.off + 255) & ~(size_t)255;
        base = cv.base ? cv.base + start : nullptr;
        state_bytes = cv.off - start;
    }

    fdtd_status carve(Carver &cv) override
    {
        const fdtd_config &c = cfg;
        geo.n[0] = c.nx;
        geo.n[1] = c.ny;
        geo.n[2] = c.nz;
        geo.px = (c.nx + 31) / 32 * 32;
        geo.PP = (long long)geo.px * c.ny;
        geo.npml = c.npml;
        for (int a = 0; a < 3; ++a) {
            geo.d0[a] = c.design_lo[a];
            geo.dn[a] = c.design_hi[a] - c.design_lo[a];
            geo.g0[a] = c.gap_lo[a];
            geo.gn[a] = c.gap_hi[a] - c.gap_lo[a];
            geo.s0[a] = c.src_lo[a];
            geo.s1[a] = c.src_hi[a];
        }
        geo.dxa = geo.d0[0] & ~3;
        geo.dp = (geo.d0[0] + geo.dn[0] - geo.dxa + 3) & ~3;
        Mdi = (long long)geo.dn[2] * geo.dn[1] * geo.dp;
        geo.Mdi = Mdi;
        geo.Mg = (int)Mg;
        geo.src_comp = c.src_comp;
        geo.sub_hi = c.sub_hi;
        geo.kappa1 = c.pml_kappa_max == 1.0;
        geo.tfsf = c.tfsf;
        for (int a = 0; a < 3; ++a) {
            geo.tf_lo[a] = c.tf_lo[a];
            geo.tf_hi[a] = c.tf_hi[a];
            if (c.tfsf) geo.s0[a] = geo.s1[a] = 0;  // the grid itself carries no source current
        }
        const long long N = c.nsteps;
        carve_state(cv, F, F_base);
        carve_state(cv, A, A_base);
        rho = cv.take<R>(Md);
        rho_t = cv.take<R>(Mdi);
        rstage = cv.take<R>(Md);
        G = cv.take<double>(Mdi);
        gstage = cv.take<double>(Md);
        gap_hist = cv.take<R>((size_t)(N + 1) * 3 * (Mg ? Mg : 1));
        const long long K = c.snapshot_every;
        rec = cv.take<R>((size_t)(K > 0 ? std::min<long long>(K, N) : N) * 3 * Mdi);
        nsnap = K > 0 ? (int)((N + K - 1) / K) : 0;
        snap_stride = snapshot_bytes<R>(c.snapshot_dtype, state_bytes);
        snaps = cv.take<char>((size_t)nsnap * snap_stride);
        src_tab = cv.take<R>(N);
        pml_tab = cv.take<R>(6 * (size_t)(c.nx + c.ny + c.nz));
        misc = cv.take<double>(4 + 2 * MMA_BLOCKS);
        err = cv.take<unsigned>(4);
        if (c.tfsf) {
            tf_tab = cv.take<R>((size_t)N * tfsf_row(geo));
            tf_col = cv.take<R>(4 * (size_t)c.nz);
        }
        nslab = (c.nz + WAVE3D_TZ - 1) / WAVE3D_TZ;
        wgx = (c.nx + WAVE3D_TX - 1) / WAVE3D_TX;
        wtpi = std::min(4, wgx);
        wipr = (wgx + wtpi - 1) / wtpi;
        wips = ((c.ny + WAVE3D_TY - 1) / WAVE3D_TY) * wipr;
        wcnt = cv.take<unsigned>(2 * (size_t)nslab + 2);
        long long njobs = 0;
        for (int k = 1; k <= WAVE_MAX; ++k) {
            wave_off[k] = njobs;
            njobs += 2LL * k * nslab;
        }
        wjobs = cv.take<int>((size_t)njobs);
        if (2LL * WAVE_MAX * nslab * wips >= (1LL << 31)) wave_req = 0;  // item index beyond int
        if (pml_tab) {
            R *t = pml_tab;
            for (int a = 0; a < 3; ++a) {
                const int n = geo.n[a];
                pm.bE[a] = t; pm.cE[a] = t + n; pm.kiE[a] = t + 2 * n;
                pm.bH[a] = t + 3 * n; pm.cH[a] = t + 4 * n; pm.kiH[a] = t + 5 * n;
                t += 6 * n;
            }
        }
        return FDTD_OK;
    }

    fdtd_status upload_tables() override
    {
        const fdtd_config &c = cfg;
        std::vector<R> tab(6 * (size_t)(c.nx + c.ny + c.nz));
        fill_pml<R>(c, c.nx, tab.data());
        fill_pml<R>(c, c.ny, tab.data() + 6 * c.nx);
        fill_pml<R>(c, c.nz, tab.data() + 6 * (c.nx + c.ny));
        std::vector<R> src = source_table<R>(c, dt);
        cudaStream_t st = stream;
        FDTD_TRY(cuda_ok(cudaMemcpyAsync(pml_tab, tab.data(), tab.size() * sizeof(R), cudaMemcpyHostToDevice, st)));
        FDTD_TRY(cuda_ok(cudaMemcpyAsync(src_tab, src.data(), src.size() * sizeof(R), cudaMemcpyHostToDevice, st)));
        launch_zero_bytes(err, 4 * sizeof(unsigned), st);
        ++launches;
        // wavefront job lists: the lag (in slabs) keeps a job's prerequisites
        // about one wave of blocks (G items) ahead of it
        wave_blocks[0] = wave3d_blocks<R>(0);
        wave_blocks[1] = wave3d_blocks<R>(1);
        {
            int dev = 0, l2 = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
            l2_budget = 0.5 * (double)l2;
            const long long G = std::max(1, std::min(wave_blocks[0], wave_blocks[1]));
            std::vector<int> all;
            for (int k = 1; k <= WAVE_MAX; ++k) {
                const long long per_key = 2LL * k * wips;
                wave_lag[k] = (int)std::max<long long>(2, 1 + (G + per_key - 1) / per_key);
                const std::vector<int> j = wave3d_jobs(nslab, k, wave_lag[k]);
                all.insert(all.end(), j.begin(), j.end());
            }
            FDTD_TRY(cuda_ok(cudaMemcpyAsync(wjobs, all.data(), all.size() * sizeof(int), cudaMemcpyHostToDevice, st)));
            launch_zero_bytes(wcnt, (size_t)(2 * nslab + 2) * sizeof(unsigned), st);
            ++launches;
        }
        if (c.tfsf) {
            // the incident wave does not depend on rho or the damping: one
            // column run per context, driven by the source plane
            Geo3D gc = geo;
            for (int a = 0; a < 3; ++a) {
                gc.s0[a] = c.src_lo[a];
                gc.s1[a] = c.src_hi[a];
            }
            const Coef<R> k = coef();
            launch_tfsf_column<R>(gc, pm, k.S, k.eps_s, k.eps_sub, src_tab, c.nsteps, tf_col, tf_tab, st);
            ++launches;
            FDTD_TRY(check_launch());
        }
        return cuda_ok(cudaStreamSynchronize(st));
    }

    Coef<R> coef() const { return make_coef<R>(cfg, dt, sigma_max, gamma_scale, terms); }

    fdtd_status forward(double *d_W) override
    {
        FDTD_TRY(cuda_ok(upload_coef_3d<R>(coef_slot, coef(), stream)));
        int f = 0, a = 0;
        FDTD_TRY(run_pass(this, 0, f, a, [&] { return enqueue_forward(); }));
        if (d_W && d_W != misc)
            FDTD_TRY(cuda_ok(cudaMemcpyAsync(d_W, misc, sizeof(double), cudaMemcpyDeviceToDevice, stream)));
        return check_launch();
    }

    fdtd_status adjoint() override
    {
        FDTD_TRY(cuda_ok(upload_coef_3d<R>(coef_slot, coef(), stream)));
        int f = 0, a = 0;
        return run_pass(this, 1, f, a, [&] { return enqueue_adjoint(); });
    }
    fdtd_status check_launch() { return cuda_ok(cudaGetLastError()); }

    fdtd_status set_design(const void *d_rho) override
    {
        cudaStream_t st = stream;
        launch_copy_check_rho<R>((const R *)d_rho, rho, Md, err, st);
        launch_pitch2d<R>(rho, rho_t, geo.dn[0], geo.dn[1] * geo.dn[2], geo.d0[0] - geo.dxa, geo.dp, st);
        launches += 2;
        FDTD_TRY(check_launch());
        unsigned h_err = 0;
        FDTD_TRY(cuda_ok(cudaMemcpyAsync(&h_err, err, sizeof(unsigned), cudaMemcpyDeviceToHost, st)));
        FDTD_TRY(cuda_ok(cudaStreamSynchronize(st)));
        if (h_err & ERR_RANGE) {
            launch_zero_bytes(err, sizeof(unsigned), st);
            cudaStreamSynchronize(st);
            return FDTD_ERANGE;
        }
        return FDTD_OK;
    }

    void advance_forward(int n0, int count, bool gap, R *rec_base)
    {
        Step3D<R> a{};
        a.rho_t = rho_t;
        if (wave_on()) {
            // runs end on multiples of the guard interval, so the guard sees
            // every step it checks
            const int T = wave_count();
            for (int n = n0; n < n0 + count;) {
                int end = n0 + count;
                if (guarding && guard_every > 0) end = std::min(end, (n / guard_every + 1) * guard_every);
                const int cnt = std::min(T, end - n);
                Wave3D<R> w = wave_plan(cnt);
                w.n0 = n;
                w.rec0 = n0;
                w.src = src_tab;
                w.gap = (gap && Mg) ? gap_hist : nullptr;
                w.rec = rec_base;
                w.tf = tf_tab;
                launches += launch_wave3d<R>(0, geo, F, coef_slot, pm, a, w, wave_blocks[0], err, WAIT_CYCLES, stream);
                cell_updates += (long long)cnt * ncells;
                n += cnt;
                if (guard_after<R>(n, F_base, state_bytes)) break;
            }
            return;
        }
        for (int n = n0; n < n0 + count; ++n) {
            a.src = src_tab + n;
            a.gap_rec = (gap && Mg) ? gap_hist + (size_t)(n + 1) * 3 * Mg : nullptr;
            a.rec = rec_base ? rec_base + (size_t)(n - n0) * 3 * Mdi : nullptr;
            a.tf_inc = tf_tab ? tf_tab + (size_t)n * tfsf_row(geo) : nullptr;
            launches += launch_step3d<R>(0, geo, F, coef_slot, pm, a, stream);
            cell_updates += ncells;
            if (guard_after<R>(n + 1, F_base, state_bytes)) break;
        }
    }

    void advance_adjoint(int m_hi, int m_lo, int slot0)
    {
        Step3D<R> a{};
        a.rho_t = rho_t;
        a.G = G;
        if (wave_on()) {
            const int T = wave_count();
            for (int m = m_hi; m > m_lo;) {
                const int cnt = std::min(T, m - m_lo);
                Wave3D<R> w = wave_plan(cnt);
                w.n0 = m;
                w.rec0 = slot0;
                w.gap = Mg ? gap_hist : nullptr;
                w.rec = rec;
                launches += launch_wave3d<R>(1, geo, A, coef_slot, pm, a, w, wave_blocks[1], err, WAIT_CYCLES, stream);
                m -= cnt;
            }
        } else {
            for (int m = m_hi; m > m_lo; --m) {
                a.gap_src = Mg ? gap_hist + (size_t)m * 3 * Mg : nullptr;
                a.rec = rec + (size_t)(m - 1 - slot0) * 3 * Mdi;
                launches += launch_step3d<R>(1, geo, A, coef_slot, pm, a, stream);
            }
        }
        cell_updates += (long long)(m_hi - m_lo) * ncells;
    }

    fdtd_status enqueue_forward()
    {
        cudaStream_t st = stream;
        const int N = cfg.nsteps, K = cfg.snapshot_every;
        launch_zero_bytes(F_base, state_bytes, st);
        if (Mg) launch_zero_bytes(gap_hist, 3 * Mg * sizeof(R), st);
        launches += 2;
        if (wave_on()) wave_reset();
        guarding = true;
        if (K <= 0) {
            advance_forward(0, N, true, rec);
        } else {
            for (int s = 0; s < nsnap; ++s) {
                if (guard_stop) break;
                const int n0 = s * K, cnt = std::min(K, N - n0);
                snapshot_save<R>(cfg.snapshot_dtype, F_base, state_bytes, snaps + (size_t)s * snap_stride, st);
                ++launches;
                advance_forward(n0, cnt, true, nullptr);
            }
        }
        guarding = false;
        if (guard_stop) return FDTD_EUNSTABLE;
        const double coefW = 0.5 * cfg.eps_g * dt * pow(cfg.dx, 3);
        launch_objective<R>(gap_hist, (long long)(N + 1) * 3 * Mg, coefW, misc, nullptr, misc + 4, err, st);
        ++launches;
        return check_launch();
    }

    fdtd_status enqueue_adjoint()
    {
        cudaStream_t st = stream;
        const int N = cfg.nsteps, K = cfg.snapshot_every;
        launch_zero_bytes(A_base, state_bytes, st);
        launch_zero_bytes(G, Mdi * sizeof(double), st);
        launches += 2;
        if (wave_on()) wave_reset();
        if (K <= 0) {
            advance_adjoint(N, 0, 0);
        } else {
            for (int s = nsnap - 1; s >= 0; --s) {
                const int n0 = s * K, n1 = std::min(n0 + K, N);
                snapshot_load<R>(cfg.snapshot_dtype, snaps + (size_t)s * snap_stride, F_base, state_bytes, st);
                ++launches;
                advance_forward(n0, n1 - n0, false, rec);
                advance_adjoint(n1, n0, n0);
            }
        }
        return check_launch();
    }

    fdtd_status gradient(double *d_grad) override
    {
        const double scale = dt * pow(cfg.dx, 3);
        launch_assemble_3d(G, d_grad, geo.dn[0], geo.dn[1], geo.dn[2], geo.d0[0] - geo.dxa, geo.dp,
                           geo.g0[0] - geo.d0[0], geo.g0[1] - geo.d0[1], geo.g0[2] - geo.d0[2], geo.gn[0], geo.gn[1],
                           geo.gn[2], scale, stream);
        ++launches;
        return check_launch();
    }

    fdtd_status grayness(double *d_zeta) override
    {
        launch_grayness<R>(rho_t, (long long)geo.dn[1] * geo.dn[2], geo.dn[0], geo.dp, geo.d0[0] - geo.dxa, geo.dn[1],
                           geo.g0[0] - geo.d0[0], geo.g0[1] - geo.d0[1], geo.g0[2] - geo.d0[2], geo.gn[0], geo.gn[1],
                           geo.gn[2], d_zeta, stream);
        launch_scale1(d_zeta, n_free > 0 ? 4.0 / (double)n_free : 0.0, stream);
        launches += 3;
        return check_launch();
    }

    fdtd_status gradient_scratch(double *d_grad, double *, double *) override { return gradient(d_grad); }

    fdtd_status gap_history(double *d_out) override
    {
        launch_to_double<R>(gap_hist, d_out, (long long)(cfg.nsteps + 1) * 3 * Mg, stream);
        ++launches;
        return check_launch();
    }
    fdtd_status gap_spectrum(const double *d_freqs, int nf, double *d_out) override
    {
        launch_gap_dft<R>(gap_hist, (long long)cfg.nsteps + 1, (int)(3 * Mg), dt, d_freqs, nf, d_out, stream);
        ++launches;
        return check_launch();
    }
};

}  // namespace

// ------------------------------------------------------------------ ABI

extern "C" {

const char *fdtd_status_string(fdtd_status s)
{
    switch (s) {
    case FDTD_OK: return "ok";
    case FDTD_EINVAL: return "invalid argument or configuration";
    case FDTD_ENOMEM: return "workspace too small";
    case FDTD_ECUDA: return "CUDA error";
    case FDTD_ESTATE: return "call out of order";
    case FDTD_EUNSTABLE: return "unstable run: non-finite objective, or a state word non-finite or above the "
                                "stability-guard bound";
    case FDTD_ETIMEOUT: return "device wait timed out";
    case FDTD_ERANGE: return "design density outside [0, 1]";
    }
    return "unknown status";
}

// Constant-memory coefficient slots of the live contexts.
static std::mutex g_slot_mu;
static bool g_slot_used[COEF_SLOTS];

static int take_slot()
{
    std::lock_guard<std::mutex> lk(g_slot_mu);
    for (int i = 0; i < COEF_SLOTS; ++i)
        if (!g_slot_used[i]) {
            g_slot_used[i] = true;
            return i;
        }
    return -1;
}

static void give_slot(int i)
{
    if (i < 0) return;
    std::lock_guard<std::mutex> lk(g_slot_mu);
    g_slot_used[i] = false;
}

static fdtd_ctx *make_ctx(const fdtd_config *cfg)
{
    fdtd_ctx *c = nullptr;
    if (cfg->ndim == 3) {
        if (cfg->real_bytes == 4) c = new (std::nothrow) Ctx3D<float>();
        else c = new (std::nothrow) Ctx3D<double>();
    } else if (cfg->pol == FDTD_POL_INPLANE) {
        if (cfg->real_bytes == 4) c = new (std::nothrow) CtxP<float>();
        else c = new (std::nothrow) CtxP<double>();
    } else {
        if (cfg->real_bytes == 4) c = new (std::nothrow) Ctx2D<float>();
        else c = new (std::nothrow) Ctx2D<double>();
    }
    if (!c) return nullptr;
    c->cfg = *cfg;
    c->dt = cfg->courant * cfg->dx / kC0;
    if (cfg->ndim == 2 && cfg->pol == FDTD_POL_INPLANE) {
        c->Md = edge_total(cfg->design_lo, cfg->design_hi);
        c->Mg = edge_total(cfg->gap_lo, cfg->gap_hi);
    } else {
        c->Md = box_count(cfg->design_lo, cfg->design_hi, cfg->ndim);
        c->Mg = box_count(cfg->gap_lo, cfg->gap_hi, cfg->ndim);
    }
    c->n_free = c->Md - c->Mg;
    c->ncells = (long long)cfg->nx * cfg->ny * (cfg->ndim == 3 ? cfg->nz : 1);
    return c;
}

fdtd_status fdtd_workspace_bytes(const fdtd_config *cfg, size_t *bytes)
{
    if (!bytes) return FDTD_EINVAL;
    FDTD_TRY(validate(cfg));
    std::unique_ptr<fdtd_ctx> c(make_ctx(cfg));
    if (!c) return FDTD_ENOMEM;
    Carver cv(nullptr);
    FDTD_TRY(c->carve(cv));
    *bytes = (cv.off + 255) & ~(size_t)255;
    return FDTD_OK;
}

fdtd_status fdtd_create(const fdtd_config *cfg, void *d_workspace, size_t bytes, void *stream, fdtd_ctx **out)
{
    if (!out || !d_workspace) return FDTD_EINVAL;
    *out = nullptr;
    FDTD_TRY(validate(cfg));
    if (((uintptr_t)d_workspace & 255) != 0) return FDTD_EINVAL;
    size_t need = 0;
    FDTD_TRY(fdtd_workspace_bytes(cfg, &need));
    if (bytes < need) return FDTD_ENOMEM;
    fdtd_ctx *c = make_ctx(cfg);
    if (!c) return FDTD_ENOMEM;
    c->coef_slot = take_slot();
    if (c->coef_slot < 0) {
        delete c;
        return FDTD_ENOMEM;
    }
    c->stream = (cudaStream_t)stream;
    c->ws = d_workspace;
    cudaGetDevice(&c->device);
    // One mapped host word for the stability guard's early stop (host
    // memory; without it the guard still reports through the error word).
    if (cudaHostAlloc((void **)&c->guard_host, sizeof(unsigned), cudaHostAllocMapped) == cudaSuccess) {
        *c->guard_host = 0;
        if (cudaHostGetDevicePointer((void **)&c->guard_host_dev, c->guard_host, 0) != cudaSuccess) {
            cudaFreeHost(c->guard_host);
            c->guard_host = c->guard_host_dev = nullptr;
        }
    } else {
        c->guard_host = nullptr;
    }
    cudaGetLastError();

    c->ws_bytes = bytes;
    Carver cv(d_workspace);
    fdtd_status s = c->carve(cv);
    if (s == FDTD_OK) s = c->upload_tables();
    if (s != FDTD_OK) {
        give_slot(c->coef_slot);
        delete c;
        return s;
    }
    *out = c;
    return FDTD_OK;
}

fdtd_status fdtd_set_design(fdtd_ctx *ctx, const void *d_rho, size_t n)
{
    if (!ctx || !d_rho || (long long)n != ctx->Md) return FDTD_EINVAL;
    ctx->has_design = ctx->fwd_done = ctx->adj_done = false;
    FDTD_TRY(ctx->set_design(d_rho));
    ctx->has_design = true;
    return FDTD_OK;
}

fdtd_status fdtd_set_damping(fdtd_ctx *ctx, double sigma_max, double gamma_scale)
{
    if (!ctx || !(sigma_max >= 0) || !(gamma_scale > 0) || !isfinite(sigma_max) || !isfinite(gamma_scale))
        return FDTD_EINVAL;
    ctx->sigma_max = sigma_max;
    ctx->gamma_scale = gamma_scale;
    ctx->fwd_done = ctx->adj_done = false;
    return FDTD_OK;
}

fdtd_status fdtd_set_stability_guard(fdtd_ctx *ctx, int every, double max_abs)
{
    if (!ctx || every < 0 || !(max_abs >= 0) || !isfinite(max_abs)) return FDTD_EINVAL;
    ctx->guard_every = every;
    ctx->guard_bound = max_abs;
    ctx->drop_graphs();  // a captured forward pass holds the old checks
    return FDTD_OK;
}

fdtd_status fdtd_set_filter_width(fdtd_ctx *ctx, double sigma)
{
    if (!ctx || !(sigma > 0) || !isfinite(sigma)) return FDTD_EINVAL;
    FDTD_TRY(ctx->set_filter_sigma(sigma));
    // rho~ = F(rho) changes: the design has to be set again
    ctx->has_design = ctx->fwd_done = ctx->adj_done = false;
    return FDTD_OK;
}

fdtd_status fdtd_set_steps_per_launch(fdtd_ctx *ctx, int steps)
{
    if (!ctx || steps < 1 || steps > 4096) return FDTD_EINVAL;
    ctx->multi_steps = steps;
    ctx->drop_graphs();  // captured passes hold the old launches
    return FDTD_OK;
}

fdtd_status fdtd_set_wavefront(fdtd_ctx *ctx, int steps)
{
    if (!ctx) return FDTD_EINVAL;
    FDTD_TRY(ctx->set_wavefront(steps));
    ctx->drop_graphs();  // captured passes hold the old launches
    return FDTD_OK;
}

fdtd_status fdtd_selftest_bounded_wait(void *d_words, long long limit_cycles, void *stream)
{
    if (!d_words || ((uintptr_t)d_words & 15) || !(limit_cycles > 0) || limit_cycles > 10000000000LL)
        return FDTD_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned *w = (unsigned *)d_words;
    launch_zero_bytes(w, 4 * sizeof(unsigned), st);
    launch_wait_selftest(w, limit_cycles, st);
    FDTD_TRY(cuda_ok(cudaGetLastError()));
    unsigned h[4] = {0, 0, 0, 0};
    FDTD_TRY(cuda_ok(cudaMemcpyAsync(h, w, sizeof h, cudaMemcpyDeviceToHost, st)));
    FDTD_TRY(cuda_ok(cudaStreamSynchronize(st)));
    if (h[2] & ERR_TIMEOUT) return h[1] ? FDTD_ETIMEOUT : FDTD_ECUDA;
    return FDTD_OK;
}

fdtd_status fdtd_set_sensitivity_terms(fdtd_ctx *ctx, int terms)
{
    if (!ctx || terms < 1 || terms > FDTD_TERM_ALL) return FDTD_EINVAL;
    ctx->terms = terms;
    ctx->adj_done = false;
    return FDTD_OK;
}

fdtd_status fdtd_forward(fdtd_ctx *ctx, double *d_W)
{
    if (!ctx) return FDTD_EINVAL;
    if (!ctx->has_design) return FDTD_ESTATE;
    ctx->fwd_done = ctx->adj_done = false;
    ctx->guard_tag = ctx->guard_tag + 1 ? ctx->guard_tag + 1 : 1;
    ctx->guard_stop = false;
    const fdtd_status s = ctx->forward(d_W);
    if (s == FDTD_EUNSTABLE) {
        // The stability guard stopped the pass: let the steps already
        // enqueued finish, then clear the error word so that the context
        // stays usable.
        cudaStreamSynchronize(ctx->stream);
        launch_zero_bytes(ctx->err_dev(), sizeof(unsigned), ctx->stream);
        ++ctx->launches;
        FDTD_TRY(cuda_ok(cudaStreamSynchronize(ctx->stream)));
        return s;
    }
    FDTD_TRY(s);
    ctx->fwd_done = true;
    return FDTD_OK;
}

fdtd_status fdtd_adjoint(fdtd_ctx *ctx)
{
    if (!ctx) return FDTD_EINVAL;
    if (!ctx->fwd_done) return FDTD_ESTATE;
    FDTD_TRY(ctx->adjoint());
    ctx->adj_done = true;
    return FDTD_OK;
}

fdtd_status fdtd_gradient(fdtd_ctx *ctx, double *d_grad, size_t n)
{
    if (!ctx || !d_grad || (long long)n != ctx->Md) return FDTD_EINVAL;
    if (!ctx->adj_done) return FDTD_ESTATE;
    return ctx->gradient(d_grad);
}

}  // extern "C"

int fdtd::context_device(const fdtd_ctx *ctx) { return ctx ? ctx->device : -1; }

int fdtd::gradient_into(fdtd_ctx *ctx, double *d_grad, size_t n, double *scratch, size_t scratch_per_array)
{
    if (!ctx || !d_grad || !scratch || (long long)n != ctx->Md) return FDTD_EINVAL;
    if (ctx->gradient_uses_scratch() && n > scratch_per_array) return FDTD_EINVAL;
    if (!ctx->adj_done) return FDTD_ESTATE;
    return ctx->gradient_scratch(d_grad, scratch, scratch + scratch_per_array);
}

extern "C" {

fdtd_status fdtd_gap_history(fdtd_ctx *ctx, double *d_out, size_t n)
{
    if (!ctx || !d_out || (long long)n != (long long)(ctx->cfg.nsteps + 1) * ctx->Mg * (ctx->cfg.ndim == 3 ? 3 : 1))
        return FDTD_EINVAL;
    if (!ctx->fwd_done) return FDTD_ESTATE;
    return ctx->gap_history(d_out);
}

fdtd_status fdtd_gap_spectrum(fdtd_ctx *ctx, const double *d_freqs, int nf, double *d_out)
{
    if (!ctx || !d_freqs || !d_out || nf < 1 || ctx->Mg < 1) return FDTD_EINVAL;
    if (!ctx->fwd_done) return FDTD_ESTATE;
    return ctx->gap_spectrum(d_freqs, nf, d_out);
}

fdtd_status fdtd_ascent_step(fdtd_ctx *ctx, void *d_rho, const double *d_grad, size_t n, double move)
{
    if (!ctx || !d_rho || !d_grad || (long long)n != ctx->Md || !(move >= 0) || !isfinite(move)) return FDTD_EINVAL;
    unsigned long long *gmax = (unsigned long long *)(ctx->W_dev() + 1);
    if (ctx->cfg.real_bytes == 4) launch_ascent<float>((float *)d_rho, d_grad, (long long)n, move, gmax, ctx->stream);
    else launch_ascent<double>((double *)d_rho, d_grad, (long long)n, move, gmax, ctx->stream);
    ctx->launches += 3;
    return cuda_ok(cudaGetLastError());
}

fdtd_status fdtd_mma_asymptotes(fdtd_ctx *ctx, const void *d_rho, const double *d_grad, double *d_state, size_t n,
                                int k, double *d_sums)
{
    if (!ctx || !d_rho || !d_grad || !d_state || !d_sums || (long long)n != ctx->Md || k < 0) return FDTD_EINVAL;
    if (ctx->cfg.real_bytes == 4)
        launch_mma_asymptotes<float>((const float *)d_rho, d_grad, d_state, (long long)n, k, ctx->W_dev() + 4, d_sums,
                                     ctx->stream);
    else
        launch_mma_asymptotes<double>((const double *)d_rho, d_grad, d_state, (long long)n, k, ctx->W_dev() + 4,
                                      d_sums, ctx->stream);
    ctx->launches += 2;
    return cuda_ok(cudaGetLastError());
}

fdtd_status fdtd_mma_solve(fdtd_ctx *ctx, const double *d_state, const double *d_grad, size_t n, double scale,
                           double raa0, double move, void *d_rho_new, double *d_sums)
{
    if (!ctx || !d_state || !d_grad || !d_rho_new || !d_sums || (long long)n != ctx->Md) return FDTD_EINVAL;
    if (!(scale > 0) || !isfinite(scale) || !(raa0 > 0) || !isfinite(raa0) || !(move > 0) || !(move <= 1))
        return FDTD_EINVAL;
    if (ctx->cfg.real_bytes == 4)
        launch_mma_solve<float>(d_state, d_grad, (long long)n, scale, raa0, move, (float *)d_rho_new,
                                ctx->W_dev() + 4, d_sums, ctx->stream);
    else
        launch_mma_solve<double>(d_state, d_grad, (long long)n, scale, raa0, move, (double *)d_rho_new,
                                 ctx->W_dev() + 4, d_sums, ctx->stream);
    ctx->launches += 2;
    return cuda_ok(cudaGetLastError());
}

static DesignRects design_rects(const fdtd_config &c)
{
    DesignRects r{};
    if (c.ndim == 2 && c.pol == FDTD_POL_INPLANE) {
        r.n = 2;
        long long off = 0;
        for (int cc = 0; cc < 2; ++cc) {
            int o[2], n[2];
            edge_rect(c.design_lo, c.design_hi, cc, o, n);
            r.off[cc] = off;
            r.w[cc] = n[0];
            r.h[cc] = n[1];
            r.d[cc] = 1;
            off += (long long)n[0] * n[1];
        }
        return r;
    }
    r.n = 1;
    r.off[0] = 0;
    r.w[0] = c.design_hi[0] - c.design_lo[0];
    r.h[0] = c.design_hi[1] - c.design_lo[1];
    r.d[0] = c.ndim == 3 ? c.design_hi[2] - c.design_lo[2] : 1;
    return r;
}

fdtd_status fdtd_mirror_average(fdtd_ctx *ctx, void *d_vec, size_t n, int elem_bytes, int axis)
{
    if (!ctx || !d_vec || (long long)n != ctx->Md || (elem_bytes != 4 && elem_bytes != 8) || axis < 0 ||
        axis >= ctx->cfg.ndim)
        return FDTD_EINVAL;
    const DesignRects r = design_rects(ctx->cfg);
    if (elem_bytes == 4) launch_mirror_avg<float>((float *)d_vec, r, axis, ctx->stream);
    else launch_mirror_avg<double>((double *)d_vec, r, axis, ctx->stream);
    ++ctx->launches;
    return cuda_ok(cudaGetLastError());
}

fdtd_status fdtd_fix_design(fdtd_ctx *ctx, void *d_rho, double *d_grad, const unsigned char *d_mask, size_t n,
                            double value)
{
    if (!ctx || !d_mask || (!d_rho && !d_grad) || (long long)n != ctx->Md || !(value >= 0.0 && value <= 1.0))
        return FDTD_EINVAL;
    if (ctx->cfg.real_bytes == 4) launch_fix<float>((float *)d_rho, d_grad, d_mask, (long long)n, value, ctx->stream);
    else launch_fix<double>((double *)d_rho, d_grad, d_mask, (long long)n, value, ctx->stream);
    ++ctx->launches;
    return cuda_ok(cudaGetLastError());
}

fdtd_status fdtd_grayness(fdtd_ctx *ctx, double *d_zeta)
{
    if (!ctx || !d_zeta) return FDTD_EINVAL;
    if (!ctx->has_design) return FDTD_ESTATE;
    return ctx->grayness(d_zeta);
}

fdtd_status fdtd_threshold(fdtd_ctx *ctx, void *d_rho, size_t n, double level)
{
    if (!ctx || !d_rho || (long long)n != ctx->Md || !isfinite(level)) return FDTD_EINVAL;
    if (ctx->cfg.real_bytes == 4) launch_threshold<float>((float *)d_rho, (long long)n, level, ctx->stream);
    else launch_threshold<double>((double *)d_rho, (long long)n, level, ctx->stream);
    ++ctx->launches;
    return cuda_ok(cudaGetLastError());
}

fdtd_status fdtd_sync(fdtd_ctx *ctx)
{
    if (!ctx) return FDTD_EINVAL;
    unsigned h = 0;
    FDTD_TRY(cuda_ok(cudaMemcpyAsync(&h, ctx->err_dev(), sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream)));
    FDTD_TRY(cuda_ok(cudaStreamSynchronize(ctx->stream)));
    if (h) {
        launch_zero_bytes(ctx->err_dev(), sizeof(unsigned), ctx->stream);
        ++ctx->launches;
        cudaStreamSynchronize(ctx->stream);
        if (h & ERR_RANGE) return FDTD_ERANGE;
        if (h & ERR_TIMEOUT) return FDTD_ETIMEOUT;
        return FDTD_EUNSTABLE;
    }
    return FDTD_OK;
}

fdtd_status fdtd_run_host(fdtd_ctx *ctx, const void *h_rho, size_t n, double *h_W, double *h_grad)
{
    if (!ctx || !h_rho || !h_W || !h_grad || (long long)n != ctx->Md) return FDTD_EINVAL;
    const size_t rb = (size_t)ctx->cfg.real_bytes;
    FDTD_TRY(cuda_ok(cudaMemcpyAsync(ctx->rho_stage(), h_rho, n * rb, cudaMemcpyHostToDevice, ctx->stream)));
    FDTD_TRY(fdtd_set_design(ctx, ctx->rho_stage(), n));
    FDTD_TRY(fdtd_forward(ctx, nullptr));
    FDTD_TRY(fdtd_adjoint(ctx));
    FDTD_TRY(fdtd_gradient(ctx, ctx->grad_stage(), n));
    FDTD_TRY(cuda_ok(cudaMemcpyAsync(h_W, ctx->W_dev(), sizeof(double), cudaMemcpyDeviceToHost, ctx->stream)));
    FDTD_TRY(cuda_ok(cudaMemcpyAsync(h_grad, ctx->grad_stage(), n * sizeof(double), cudaMemcpyDeviceToHost,
                                     ctx->stream)));
    return fdtd_sync(ctx);
}

fdtd_status fdtd_get_info(const fdtd_ctx *ctx, fdtd_info *info)
{
    if (!ctx || !info) return FDTD_EINVAL;
    info->dt = ctx->dt;
    info->n_cells = ctx->ncells;
    info->n_design = ctx->Md;
    info->n_gap = ctx->Mg;
    info->launches = ctx->launches;
    info->cell_updates = ctx->cell_updates;
    info->workspace_bytes = ctx->ws_bytes;
    ctx->block_counts(&info->step_blocks, &info->vector_blocks);
    return FDTD_OK;
}

void fdtd_destroy(fdtd_ctx *ctx)
{
    if (!ctx) return;
    give_slot(ctx->coef_slot);
    delete ctx;
}

fdtd_status fdtd_set_l2_residency(fdtd_ctx *ctx, double fraction)
{
    if (!ctx || !(fraction >= 0.0 && fraction <= 1.0)) return FDTD_EINVAL;
    return ctx->set_l2(fraction);
}

fdtd_status fdtd_set_graphs(fdtd_ctx *ctx, int mode)
{
    if (!ctx || mode < 0 || mode > 2) return FDTD_EINVAL;
    ctx->graphs = mode;
    return FDTD_OK;
}

}  // extern "C"
