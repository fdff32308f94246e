/*
 * fdtd_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU restatement of the hot path of Hassan & Cala Lesina,
 * "Topology optimization of dispersive plasmonic nanostructures in the
 * time-domain" (arXiv 2203.01462).  It exists to check the CUDA library: only
 * the tests, the smoke check and the benchmark's CPU-baseline leg load it.  It
 * shares no code, header, table or constant generator with the CUDA library,
 * and the product path never calls it.
 *
 * Every quantity is in SI units.  The steps follow the paper in its order:
 *
 *   Sec. 2.1, Eq. (5a-c)  rho_i -> eps_inf_i, psi_i, sigma_i (linear in rho for
 *                         eps_inf and psi = omega_p^2, parabolic sigma).
 *   Sec. 3.1, Eq. (10)    eps0 eps_inf dE/dt + J + sigma E - curl H = -J_src
 *                         dJ/dt + gamma J - eps0 psi E = 0
 *                         mu0 dH/dt + curl E = 0
 *   Sec. 3.2              Yee grid, E (and J) at integer steps, H at half
 *                         steps.  The paper says it uses the ADE approach but
 *                         prints no update; the reading taken here is a
 *                         trapezoidal average of J and sigma E over the step,
 *                         so that each node solves a 2x2 linear system.
 *                         Open boundaries: CPML (Roden-Gedney recursive
 *                         convolution), PEC walls behind it.
 *   Eq. (24)              W~ = eps_g dt dx^d / 2 * sum_{n=0..N} sum_gap (E^n)^2
 *                         (d = 2 in 2D, i.e. per unit length in z).
 *   Eq. (20)              adjoint run: the same solver, started from rest,
 *                         driven by eps_g E(T - tau) in the gap; its E*, J*
 *                         live at half steps.
 *   Eq. (25a-c)           pointwise sensitivities, sums over n = 0..N of
 *                         E_i^{N-n} times half-step averages / differences of
 *                         the adjoint fields (E*^{-1/2} = J*^{-1/2} = 0).
 *   Eq. (26), (27)        filtered design rho~ = F(rho) and the chain rule.
 *                         F is a normalised Gaussian; the chain rule applies
 *                         F^T (the paper writes the diagonal d rho~_i/d rho_i).
 *
 * 3D plane wave (Sec. 3.3 injects one at normal incidence): total-field /
 * scattered-field, with the incident field taken from a 1D column of the
 * same scheme (see the 3D part below).
 *
 * The oracle keeps whole arrays (no slabs), loops node by node and solves
 * each node's 2x2 system by Cramer's rule.  Loops over nodes may run under
 * OpenMP; every per-node result and every sum is formed in a fixed order, so
 * results do not depend on the thread count.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* CODATA 2018 values. */
#define OR_C0 299792458.0
#define OR_MU0 1.25663706212e-6
#define OR_PI 3.14159265358979323846

typedef struct or_config {
    int ndim;              /* 2: TM_z (Ez, Hx, Hy, Jz); 3: full Yee            */
    int nx, ny, nz;        /* nodes (2D) / cells (3D) per axis                  */
    double dx;             /* grid step, m                                      */
    double courant;        /* S = c0 dt / dx                                    */
    int npml;              /* CPML layers on each open side; 0 = PEC walls      */
    double pml_m;          /* polynomial grading order                          */
    double pml_sigma_factor; /* sigma_pml_max = factor (m+1) / (eta0 dx)         */
    double pml_kappa_max;
    double pml_alpha_max;  /* S/m, linear taper to 0 at the outer wall          */
    int periodic_x;        /* 2D: x is periodic (no walls, no CPML in x)        */
    double eps_inf, omega_p, gamma_p; /* Drude material, Eq. (1)                */
    double eps_s;          /* background relative permittivity                  */
    double psi_s_ratio;    /* psi_s = ratio * omega_p^2 (the paper uses 1/100)  */
    double eps_g;          /* gap (observation region) permittivity             */
    int design_lo[3], design_hi[3]; /* design box, half-open node/cell ranges   */
    int gap_lo[3], gap_hi[3];       /* gap box (inside the design box)          */
    int src_lo[3], src_hi[3];       /* soft current source box (Ez nodes/edges) */
    int nbands;            /* 1 or 2 carriers under one envelope                */
    double f0[2];          /* carrier frequencies, Hz                           */
    double tau, t0;        /* Gaussian envelope exp(-((t-t0)/tau)^2), s         */
    double src_amp;        /* J_src = src_amp * eps0 c0 / dx * g(t), A/m^2      */
    int nsteps;            /* N: E^0 .. E^N                                     */
    int filter_radius;     /* Gaussian filter half-width in cells; 0 = none     */
    double filter_sigma;   /* Gaussian filter standard deviation in cells       */
    int sigma_form;        /* 0: rho(1-rho) smax (Eq. 5c); 1: 4 rho(1-rho) smax */
    double sub_eps;        /* 3D: background eps for cells with k < sub_hi      */
    int sub_hi;
    int src_comp;          /* 3D: component driven by the source (0 x, 1 y, 2 z) */
    int waveform;          /* 0: Gaussian envelope; 1: truncated sinc x Hanning */
    double bandwidth;      /* waveform 1: width B of the rectangular spectrum, Hz */
    int lobes;             /* waveform 1: sinc kept for |t - t0| < lobes / B     */
    int pol;               /* 2D: 0 = E_z out of plane (Ez, Hx, Hy, Jz);        */
                           /* 1 = E in plane (Ex, Ey, Hz, Jx, Jy), design and   */
                           /* gap per Yee edge                                  */
    int tfsf;              /* 3D: 1 = plane wave by total-field / scattered-    */
                           /* field injection instead of the source box         */
    int tf_lo[3], tf_hi[3]; /* total-field region: the closed box of positions  */
                           /* tf_lo <= x <= tf_hi (node units)                  */
} or_config;

static int g_threads = 1;

void or_set_threads(int n)
{
    g_threads = n < 1 ? 1 : n;
#ifdef _OPENMP
    omp_set_num_threads(g_threads);
#endif
}

int or_get_threads(void) { return g_threads; }

static double or_eps0(void) { return 1.0 / (OR_MU0 * OR_C0 * OR_C0); }
static double or_dt(const or_config *c) { return c->courant * c->dx / OR_C0; }

/* Excitation: carrier(s) sin(2 pi f0 (t - t0)) under an envelope.
 * waveform 0: Gaussian exp(-((t - t0)/tau)^2).
 * waveform 1 (the paper's, Sec. 2 and Fig. 1c-d): a sinc whose spectrum is
 * a rectangle of width B, sin(pi B u)/(pi B u) with u = t - t0, truncated
 * after `lobes` lobes on each side (|u| < T = lobes/B) and smoothed by the
 * Hanning window (1 + cos(pi u / T))/2, which rounds the spectrum's edges. */
static double or_signal(const or_config *c, double t)
{
    const double u = t - c->t0;
    double s = 0.0;
    for (int b = 0; b < c->nbands; ++b)
        s += sin(2.0 * OR_PI * c->f0[b] * u);
    if (c->waveform == 1) {
        const double T = c->lobes / c->bandwidth;
        if (fabs(u) >= T) return 0.0;
        const double x = OR_PI * c->bandwidth * u;
        const double sinc = x == 0.0 ? 1.0 : sin(x) / x;
        return sinc * 0.5 * (1.0 + cos(OR_PI * u / T)) * s;
    }
    return exp(-(u / c->tau) * (u / c->tau)) * s;
}

/* The excitation sampled at times t (n samples), for tests. */
void or_signal_samples(const or_config *c, const double *t, int n, double *out)
{
    for (int k = 0; k < n; ++k) out[k] = or_signal(c, t[k]);
}

/* Eq. (5a-c): material of one design node from its filtered density. */
void or_material(const or_config *c, double rho, double sigma_max,
                 double *eps_i, double *psi_i, double *sig_i)
{
    double psi = c->omega_p * c->omega_p;
    double psi_s = c->psi_s_ratio * psi;
    *eps_i = c->eps_s + rho * (c->eps_inf - c->eps_s);
    *psi_i = psi_s + rho * (psi - psi_s);
    *sig_i = rho * (1.0 - rho) * sigma_max * (c->sigma_form ? 4.0 : 1.0);
}

/* ---------------------------------------------------------------- boxes */

static int in_box(const int *lo, const int *hi, int i, int j, int k)
{
    return i >= lo[0] && i < hi[0] && j >= lo[1] && j < hi[1] && k >= lo[2] && k < hi[2];
}

static long box_count(const int *lo, const int *hi, int ndim)
{
    long n = 1;
    for (int a = 0; a < ndim; ++a) {
        if (hi[a] <= lo[a]) return 0;
        n *= hi[a] - lo[a];
    }
    return n;
}

/* In-plane 2D (pol 1): the design and gap boxes are cell ranges; their
 * Yee edges are E_x edges (i+1/2, j) with lo_x <= i < hi_x, lo_y <= j <= hi_y
 * and E_y edges (i, j+1/2) with lo_x <= i <= hi_x, lo_y <= j < hi_y. */
static long edge_count(const int *lo, const int *hi)
{
    long w = hi[0] - lo[0], h = hi[1] - lo[1];
    if (w <= 0 || h <= 0) return 0;
    return w * (h + 1) + (w + 1) * h;
}

int or_sizes(const or_config *c, long *n_design, long *n_gap)
{
    if (c->ndim == 2 && c->pol == 1) {
        *n_design = edge_count(c->design_lo, c->design_hi);
        *n_gap = edge_count(c->gap_lo, c->gap_hi);
        return 0;
    }
    *n_design = box_count(c->design_lo, c->design_hi, c->ndim);
    *n_gap = box_count(c->gap_lo, c->gap_hi, c->ndim);
    return 0;
}

/* Index of an edge within the edge list of a cell box (E_x edges first, row
 * by row, then E_y edges), or -1 if the edge is not in the box's set. */
static long edge_index(const int *lo, const int *hi, int comp, int i, int j)
{
    long w = hi[0] - lo[0], h = hi[1] - lo[1];
    if (comp == 0) {
        if (i < lo[0] || i >= hi[0] || j < lo[1] || j > hi[1]) return -1;
        return (long)(j - lo[1]) * w + (i - lo[0]);
    }
    if (i < lo[0] || i > hi[0] || j < lo[1] || j >= hi[1]) return -1;
    return w * (h + 1) + (long)(j - lo[1]) * (w + 1) + (i - lo[0]);
}

/* Free design variables: design edges outside the gap (the counts of Sec. 3.2). */
long or_free_design(const or_config *c)
{
    long M, G;
    or_sizes(c, &M, &G);
    if (c->ndim == 2 && c->pol == 1) {
        long n = 0;
        for (int comp = 0; comp < 2; ++comp)
            for (int j = c->design_lo[1]; j <= c->design_hi[1]; ++j)
                for (int i = c->design_lo[0]; i <= c->design_hi[0]; ++i)
                    if (edge_index(c->design_lo, c->design_hi, comp, i, j) >= 0 &&
                        edge_index(c->gap_lo, c->gap_hi, comp, i, j) < 0)
                        ++n;
        return n;
    }
    return M - G;
}

/* ------------------------------------------------------------- filter */

/* Eq. (26): rho~ = F(rho), F a Gaussian window of half-width R cells,
 * weights renormalised where the window leaves the design box.  Written as
 * the plain double (2D) or triple (3D) sum. */
static void filter_apply(const or_config *c, const double *in, double *out, int transpose)
{
    int w = c->design_hi[0] - c->design_lo[0];
    int h = c->design_hi[1] - c->design_lo[1];
    int d = c->ndim == 3 ? c->design_hi[2] - c->design_lo[2] : 1;
    int R = c->filter_radius;
    long M = (long)w * h * d;
    if (R <= 0) {
        memcpy(out, in, sizeof(double) * M);
        return;
    }
    double s2 = 2.0 * c->filter_sigma * c->filter_sigma;
    int Rz = c->ndim == 3 ? R : 0;
    double *norm = (double *)malloc(sizeof(double) * M);
    for (int z = 0; z < d; ++z)
        for (int y = 0; y < h; ++y)
            for (int x = 0; x < w; ++x) {
                double s = 0.0;
                for (int dz = -Rz; dz <= Rz; ++dz)
                    for (int dy = -R; dy <= R; ++dy)
                        for (int dx = -R; dx <= R; ++dx) {
                            int xx = x + dx, yy = y + dy, zz = z + dz;
                            if (xx < 0 || xx >= w || yy < 0 || yy >= h || zz < 0 || zz >= d) continue;
                            s += exp(-(dx * dx + dy * dy + dz * dz) / s2);
                        }
                norm[((long)z * h + y) * w + x] = s;
            }
    for (long m = 0; m < M; ++m) out[m] = 0.0;
    for (int z = 0; z < d; ++z)
        for (int y = 0; y < h; ++y)
            for (int x = 0; x < w; ++x) {
                long i = ((long)z * h + y) * w + x;
                double acc = 0.0;
                for (int dz = -Rz; dz <= Rz; ++dz)
                    for (int dy = -R; dy <= R; ++dy)
                        for (int dx = -R; dx <= R; ++dx) {
                            int xx = x + dx, yy = y + dy, zz = z + dz;
                            if (xx < 0 || xx >= w || yy < 0 || yy >= h || zz < 0 || zz >= d) continue;
                            long j = ((long)zz * h + yy) * w + xx;
                            double wij = exp(-(dx * dx + dy * dy + dz * dz) / s2);
                            if (!transpose)
                                acc += wij * in[j];           /* row i of F times rho   */
                            else
                                out[j] += wij / norm[i] * in[i]; /* column i of F^T    */
                        }
                if (!transpose) out[i] = acc / norm[i];
            }
    free(norm);
}

void or_filter(const or_config *c, const double *in, double *out) { filter_apply(c, in, out, 0); }
void or_filter_T(const or_config *c, const double *in, double *out) { filter_apply(c, in, out, 1); }

/* --------------------------------------------------------------- CPML */

/* Depth (in cells) of a position p (in cell units) inside the absorbing
 * layer of an axis with n nodes; 0 in the interior. */
static double pml_depth(const or_config *c, int n, double p)
{
    double L = c->npml;
    if (c->npml <= 0) return 0.0;
    if (p < L) return L - p;
    if (p > (n - 1) - L) return p - ((n - 1) - L);
    return 0.0;
}

typedef struct { double b, c, kappa; } pml_coef;

/* Roden-Gedney CPML: sigma, kappa polynomially graded, alpha linear. */
static pml_coef pml_at(const or_config *c, int n, double p)
{
    pml_coef r = {0.0, 0.0, 1.0};
    double d = pml_depth(c, n, p);
    if (d <= 0.0) return r;
    double eps0 = or_eps0();
    double eta0 = OR_MU0 * OR_C0;
    double x = d / c->npml;
    double xm = pow(x, c->pml_m);
    double smax = c->pml_sigma_factor * (c->pml_m + 1.0) / (eta0 * c->dx);
    double sig = smax * xm;
    double kap = 1.0 + (c->pml_kappa_max - 1.0) * xm;
    double alp = c->pml_alpha_max * (1.0 - x);
    r.kappa = kap;
    r.b = exp(-(sig / kap + alp) * or_dt(c) / eps0);
    r.c = sig > 0.0 ? sig / (sig * kap + kap * kap * alp) * (r.b - 1.0) : 0.0;
    return r;
}

/* ------------------------------------------------------- node solve */

/* One node of Eq. (10a,b) over one step, trapezoidal in J and sigma E:
 *   eps0 eps (E'-E)/dt + (J'+J)/2 + sig (E'+E)/2 = curl - jsrc
 *   (J'-J)/dt + gam (J'+J)/2 = eps0 psi (E'+E)/2
 * solved for (E', J') by Cramer's rule. */
static void node_solve(double eps, double psi, double sig, double gam, double dt,
                       double curl, double jsrc, double *E, double *J)
{
    double eps0 = or_eps0();
    double a11 = eps0 * eps / dt + 0.5 * sig, a12 = 0.5;
    double a21 = -0.5 * eps0 * psi, a22 = 1.0 / dt + 0.5 * gam;
    double b1 = (eps0 * eps / dt - 0.5 * sig) * (*E) - 0.5 * (*J) + curl - jsrc;
    double b2 = (1.0 / dt - 0.5 * gam) * (*J) + 0.5 * eps0 * psi * (*E);
    double det = a11 * a22 - a12 * a21;
    *E = (b1 * a22 - a12 * b2) / det;
    *J = (a11 * b2 - a21 * b1) / det;
}

/* ================================================================ 2D */

typedef struct {
    int nx, ny;
    double *Ez, *Jz, *Hx, *Hy;
    double *pezx, *pezy, *phxy, *phyx;   /* CPML convolution terms */
} st2;

typedef struct {
    double *eps, *psi, *sig;             /* per Ez node */
    double gam;                          /* Drude collision rate (scaled) */
    pml_coef *ex, *ey, *hx, *hy;         /* CPML at E / H positions per axis */
} mat2;

static void st2_alloc(st2 *s, int nx, int ny)
{
    size_t n = (size_t)nx * ny;
    s->nx = nx; s->ny = ny;
    s->Ez = calloc(n, sizeof(double)); s->Jz = calloc(n, sizeof(double));
    s->Hx = calloc(n, sizeof(double)); s->Hy = calloc(n, sizeof(double));
    s->pezx = calloc(n, sizeof(double)); s->pezy = calloc(n, sizeof(double));
    s->phxy = calloc(n, sizeof(double)); s->phyx = calloc(n, sizeof(double));
}

static void st2_free(st2 *s)
{
    free(s->Ez); free(s->Jz); free(s->Hx); free(s->Hy);
    free(s->pezx); free(s->pezy); free(s->phxy); free(s->phyx);
}

/* Material of every Ez node.  Outside the design box: background eps_s.
 * Design box: Eq. (5a-c) from the filtered density.  Gap: eps_g, no Drude. */
static void mat2_build(const or_config *c, const double *rho_t, double sigma_max,
                       double gamma_scale, mat2 *m)
{
    int nx = c->nx, ny = c->ny;
    size_t n = (size_t)nx * ny;
    m->eps = malloc(n * sizeof(double));
    m->psi = calloc(n, sizeof(double));
    m->sig = calloc(n, sizeof(double));
    m->gam = c->gamma_p * gamma_scale;
    int w = c->design_hi[0] - c->design_lo[0];
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t q = (size_t)j * nx + i;
            m->eps[q] = c->eps_s;
            if (in_box(c->gap_lo, c->gap_hi, i, j, 0)) {
                m->eps[q] = c->eps_g;
            } else if (in_box(c->design_lo, c->design_hi, i, j, 0)) {
                double r = rho_t[(size_t)(j - c->design_lo[1]) * w + (i - c->design_lo[0])];
                or_material(c, r, sigma_max, &m->eps[q], &m->psi[q], &m->sig[q]);
            }
        }
    m->ex = malloc(nx * sizeof(pml_coef)); m->hx = malloc(nx * sizeof(pml_coef));
    m->ey = malloc(ny * sizeof(pml_coef)); m->hy = malloc(ny * sizeof(pml_coef));
    or_config cx = *c;
    if (c->periodic_x) cx.npml = 0;
    for (int i = 0; i < nx; ++i) { m->ex[i] = pml_at(&cx, nx, i); m->hx[i] = pml_at(&cx, nx, i + 0.5); }
    for (int j = 0; j < ny; ++j) { m->ey[j] = pml_at(c, ny, j); m->hy[j] = pml_at(c, ny, j + 0.5); }
}

static void mat2_free(mat2 *m)
{
    free(m->eps); free(m->psi); free(m->sig);
    free(m->ex); free(m->ey); free(m->hx); free(m->hy);
}


/* H half of one leapfrog step (2D TM_z): mu0 dH/dt = -curl E, so
 * H^{n-1/2} -> H^{n+1/2} from E^n, with the CPML terms of each derivative. */
static void step2_h(const or_config *c, const mat2 *m, st2 *s)
{
    int nx = c->nx, ny = c->ny, per = c->periodic_x;
    double dx = c->dx, ch = or_dt(c) / OR_MU0;
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            size_t q = (size_t)j * nx + i;
            if (j + 1 < ny) {
                double dEy = (s->Ez[q + nx] - s->Ez[q]) / dx;
                s->phxy[q] = m->hy[j].b * s->phxy[q] + m->hy[j].c * dEy;
                s->Hx[q] -= ch * (dEy / m->hy[j].kappa + s->phxy[q]);
            }
            int ip = i + 1;
            if (ip == nx) {
                if (!per) continue;
                ip = 0;
            }
            double dEx = (s->Ez[(size_t)j * nx + ip] - s->Ez[q]) / dx;
            s->phyx[q] = m->hx[i].b * s->phyx[q] + m->hx[i].c * dEx;
            s->Hy[q] += ch * (dEx / m->hx[i].kappa + s->phyx[q]);
        }
    }
}

/* E, J half of one leapfrog step (2D TM_z): Eq. (10a,b) at every Ez node,
 * driven by the current density jsrc (per node, taken at n+1/2).  With PEC
 * walls the outermost Ez nodes stay zero; with periodic x every column is
 * updated and indices wrap. */
static void step2_e(const or_config *c, const mat2 *m, st2 *s, const double *jsrc)
{
    int nx = c->nx, ny = c->ny, per = c->periodic_x;
    double dt = or_dt(c), dx = c->dx;
    #pragma omp parallel for schedule(static)
    for (int j = 1; j < ny - 1; ++j) {
        for (int i = 0; i < nx; ++i) {
            if (!per && (i == 0 || i == nx - 1)) continue;
            int im = i == 0 ? nx - 1 : i - 1;
            size_t q = (size_t)j * nx + i;
            double dHy = (s->Hy[q] - s->Hy[(size_t)j * nx + im]) / dx;
            double dHx = (s->Hx[q] - s->Hx[q - nx]) / dx;
            s->pezx[q] = m->ex[i].b * s->pezx[q] + m->ex[i].c * dHy;
            s->pezy[q] = m->ey[j].b * s->pezy[q] + m->ey[j].c * dHx;
            double curl = dHy / m->ex[i].kappa + s->pezx[q] - dHx / m->ey[j].kappa - s->pezy[q];
            node_solve(m->eps[q], m->psi[q], m->sig[q], m->gam, dt, curl,
                       jsrc[q], &s->Ez[q], &s->Jz[q]);
        }
    }
}

/* Discrete electromagnetic energy (per unit length in z) at step n from E^n
 * and the H half steps on either side: sum eps0 eps (E^n)^2 / 2 +
 * mu0 H^{n-1/2} . H^{n+1/2} / 2, times dx^2.  Lossless media conserve it. */
static double energy2(const or_config *c, const mat2 *m, const st2 *s,
                      const double *Hx_old, const double *Hy_old)
{
    double eps0 = or_eps0(), e = 0.0;
    size_t n = (size_t)c->nx * c->ny;
    for (size_t q = 0; q < n; ++q) {
        e += 0.5 * eps0 * m->eps[q] * s->Ez[q] * s->Ez[q];
        e += 0.5 * OR_MU0 * (Hx_old[q] * s->Hx[q] + Hy_old[q] * s->Hy[q]);
    }
    return e * c->dx * c->dx;
}

/* Forward solve (2D).  Records E^n, n = 0..N, in the gap and the design box,
 * optional probes and an optional energy trace (entries 0..N-1), and returns
 * W~ of Eq. (24). */
static int forward2(const or_config *c, const double *rho, double sigma_max, double gamma_scale,
                    double *W, double *gap_hist, double *design_hist,
                    const int *probes, int nprobe, double *probe_hist, double *energy)
{
    int nx = c->nx, N = c->nsteps;
    long M, G;
    or_sizes(c, &M, &G);
    double *rho_t = malloc(sizeof(double) * (M ? M : 1));
    if (M) or_filter(c, rho, rho_t);
    mat2 m;
    mat2_build(c, rho_t, sigma_max, gamma_scale, &m);
    st2 s;
    st2_alloc(&s, nx, c->ny);
    size_t n = (size_t)nx * c->ny;
    double *jsrc = calloc(n, sizeof(double));
    double *hxo = energy ? calloc(n, sizeof(double)) : NULL;
    double *hyo = energy ? calloc(n, sizeof(double)) : NULL;
    double dt = or_dt(c);
    double J0 = c->src_amp * or_eps0() * OR_C0 / c->dx;
    double sum = 0.0;
    int gw = c->gap_hi[0] - c->gap_lo[0];
    int dw = c->design_hi[0] - c->design_lo[0];

    for (int t = 0; t <= N; ++t) {
        for (int j = c->gap_lo[1]; j < c->gap_hi[1]; ++j)
            for (int i = c->gap_lo[0]; i < c->gap_hi[0]; ++i) {
                double e = s.Ez[(size_t)j * nx + i];
                sum += e * e;
                if (gap_hist)
                    gap_hist[(size_t)t * G + (size_t)(j - c->gap_lo[1]) * gw + (i - c->gap_lo[0])] = e;
            }
        if (design_hist)
            for (int j = c->design_lo[1]; j < c->design_hi[1]; ++j)
                for (int i = c->design_lo[0]; i < c->design_hi[0]; ++i)
                    design_hist[(size_t)t * M + (size_t)(j - c->design_lo[1]) * dw + (i - c->design_lo[0])] =
                        s.Ez[(size_t)j * nx + i];
        for (int p = 0; p < nprobe; ++p)
            probe_hist[(size_t)t * nprobe + p] = s.Ez[(size_t)probes[2 * p + 1] * nx + probes[2 * p]];
        if (t == N) break;
        double js = J0 * or_signal(c, (t + 0.5) * dt);
        for (int j = c->src_lo[1]; j < c->src_hi[1]; ++j)
            for (int i = c->src_lo[0]; i < c->src_hi[0]; ++i)
                jsrc[(size_t)j * nx + i] = js;
        if (energy) {
            memcpy(hxo, s.Hx, n * sizeof(double));
            memcpy(hyo, s.Hy, n * sizeof(double));
        }
        step2_h(c, &m, &s);
        if (energy) energy[t] = energy2(c, &m, &s, hxo, hyo);
        step2_e(c, &m, &s, jsrc);
    }
    *W = 0.5 * c->eps_g * dt * c->dx * c->dx * sum;
    free(jsrc); free(hxo); free(hyo); free(rho_t);
    st2_free(&s);
    mat2_free(&m);
    return 0;
}

/* Forward, adjoint and gradient (2D).
 *
 * Adjoint (Eq. 20): the forward solver, from rest, with the source term
 * eps_g E(T - tau) in the gap.  The forward solver takes its source as
 * -J_src on the right of Ampere's law, so the adjoint passes
 * J_src = -eps_g E^{N-n} at adjoint step n, n = 0..N; step n turns
 * E*^{n-1/2} into E*^{n+1/2} (and J* likewise).
 *
 * Sensitivities (Eq. 25a-c), per design node i outside the gap:
 *   dW/dpsi_i     = -(dt dx^2 / psi_i) sum_n E_i^{N-n} (J*^{n+1/2} + J*^{n-1/2}) / 2
 *   dW/deps_inf_i = -eps0 dx^2        sum_n E_i^{N-n} (E*^{n+1/2} - E*^{n-1/2})
 *   dW/dsigma_i   = -dt dx^2          sum_n E_i^{N-n} (E*^{n+1/2} + E*^{n-1/2}) / 2
 * Chain rule (Eq. 27) with d psi_i/d rho~ = psi - psi_s,
 * d eps_inf_i/d rho~ = eps_inf - eps_s, d sigma_i/d rho~ = smax (1 - 2 rho~)
 * (times 4 for the peak-normalised form), zero in the gap, then F^T, then
 * zero in the gap again (gap densities are not design variables). */
static int gradient2(const or_config *c, const double *rho, double sigma_max, double gamma_scale,
                     double *W, double *grad, double *g_psi, double *g_eps, double *g_sig)
{
    int nx = c->nx, N = c->nsteps;
    long M, G;
    or_sizes(c, &M, &G);
    if (M == 0) return -1;
    double *ghist = malloc(sizeof(double) * (size_t)(N + 1) * (G ? G : 1));
    double *dhist = malloc(sizeof(double) * (size_t)(N + 1) * M);
    forward2(c, rho, sigma_max, gamma_scale, W, ghist, dhist, NULL, 0, NULL, NULL);

    double *rho_t = malloc(sizeof(double) * M);
    or_filter(c, rho, rho_t);
    mat2 m;
    mat2_build(c, rho_t, sigma_max, gamma_scale, &m);
    st2 a;
    st2_alloc(&a, nx, c->ny);
    size_t n = (size_t)nx * c->ny;
    double *jsrc = calloc(n, sizeof(double));
    double *sp = calloc(M, sizeof(double)), *se = calloc(M, sizeof(double)), *ss = calloc(M, sizeof(double));
    double *Eold = malloc(sizeof(double) * M), *Jold = malloc(sizeof(double) * M);
    int dw = c->design_hi[0] - c->design_lo[0];
    int gw = c->gap_hi[0] - c->gap_lo[0];

    for (int t = 0; t <= N; ++t) {
        for (int j = c->gap_lo[1]; j < c->gap_hi[1]; ++j)
            for (int i = c->gap_lo[0]; i < c->gap_hi[0]; ++i)
                jsrc[(size_t)j * nx + i] =
                    -c->eps_g * ghist[(size_t)(N - t) * G + (size_t)(j - c->gap_lo[1]) * gw + (i - c->gap_lo[0])];
        for (int j = c->design_lo[1]; j < c->design_hi[1]; ++j)
            for (int i = c->design_lo[0]; i < c->design_hi[0]; ++i) {
                long d = (long)(j - c->design_lo[1]) * dw + (i - c->design_lo[0]);
                Eold[d] = a.Ez[(size_t)j * nx + i];
                Jold[d] = a.Jz[(size_t)j * nx + i];
            }
        step2_h(c, &m, &a);
        step2_e(c, &m, &a, jsrc);
        for (int j = c->design_lo[1]; j < c->design_hi[1]; ++j)
            for (int i = c->design_lo[0]; i < c->design_hi[0]; ++i) {
                long d = (long)(j - c->design_lo[1]) * dw + (i - c->design_lo[0]);
                double Ef = dhist[(size_t)(N - t) * M + d];
                double En = a.Ez[(size_t)j * nx + i], Jn = a.Jz[(size_t)j * nx + i];
                sp[d] += Ef * 0.5 * (Jn + Jold[d]);
                se[d] += Ef * (En - Eold[d]);
                ss[d] += Ef * 0.5 * (En + Eold[d]);
            }
    }

    double eps0 = or_eps0(), dt = or_dt(c), dx2 = c->dx * c->dx;
    double psi = c->omega_p * c->omega_p, psi_s = c->psi_s_ratio * psi;
    double *gt = malloc(sizeof(double) * M);
    for (int j = c->design_lo[1]; j < c->design_hi[1]; ++j)
        for (int i = c->design_lo[0]; i < c->design_hi[0]; ++i) {
            long d = (long)(j - c->design_lo[1]) * dw + (i - c->design_lo[0]);
            double ep, ps, sg;
            or_material(c, rho_t[d], sigma_max, &ep, &ps, &sg);
            double dpsi = -(dt * dx2 / ps) * sp[d];
            double deps = -eps0 * dx2 * se[d];
            double dsig = -dt * dx2 * ss[d];
            if (in_box(c->gap_lo, c->gap_hi, i, j, 0)) dpsi = deps = dsig = 0.0;
            if (g_psi) g_psi[d] = dpsi;
            if (g_eps) g_eps[d] = deps;
            if (g_sig) g_sig[d] = dsig;
            double dsdr = sigma_max * (1.0 - 2.0 * rho_t[d]) * (c->sigma_form ? 4.0 : 1.0);
            gt[d] = (psi - psi_s) * dpsi + (c->eps_inf - c->eps_s) * deps + dsdr * dsig;
        }
    or_filter_T(c, gt, grad);
    for (int j = c->gap_lo[1]; j < c->gap_hi[1]; ++j)
        for (int i = c->gap_lo[0]; i < c->gap_hi[0]; ++i)
            grad[(long)(j - c->design_lo[1]) * dw + (i - c->design_lo[0])] = 0.0;

    free(gt); free(Eold); free(Jold); free(sp); free(se); free(ss);
    free(jsrc); free(rho_t); free(ghist); free(dhist);
    st2_free(&a);
    mat2_free(&m);
    return 0;
}

/* ===================================================== 2D, E in plane */

/* Grid of nx x ny nodes: Ex(i,j) on the edge (i+1/2, j), Ey(i,j) on
 * (i, j+1/2), Hz(i,j) at the cell centre (i+1/2, j+1/2); Drude Jx, Jy on the
 * edges of the design box.  This is the paper's 2D "TM" case (H out of
 * plane, E in plane, surface plasmons possible; Sec. 3.2 names it with H_x
 * and E_y, E_z in the y-z plane).  PEC walls: Ex vanishes on the rows j = 0
 * and ny-1, Ey on the columns i = 0 and nx-1; with periodic x every column
 * is updated and x indices wrap. */
typedef struct {
    double *Ex, *Ey, *Jx, *Jy, *Hz;
    double *pexy, *peyx, *phzx, *phzy;   /* CPML terms: Ex d/dy, Ey d/dx, Hz d/dx, Hz d/dy */
} st2t;

typedef struct {
    double *eps[2], *psi[2], *sig[2];    /* per edge, component 0 = x, 1 = y */
    double gam;
    pml_coef *ex, *ey, *hx, *hy;
} mat2t;

static void st2t_alloc(const or_config *c, st2t *s)
{
    size_t n = (size_t)c->nx * c->ny;
    s->Ex = calloc(n, sizeof(double)); s->Ey = calloc(n, sizeof(double));
    s->Jx = calloc(n, sizeof(double)); s->Jy = calloc(n, sizeof(double));
    s->Hz = calloc(n, sizeof(double));
    s->pexy = calloc(n, sizeof(double)); s->peyx = calloc(n, sizeof(double));
    s->phzx = calloc(n, sizeof(double)); s->phzy = calloc(n, sizeof(double));
}

static void st2t_free(st2t *s)
{
    free(s->Ex); free(s->Ey); free(s->Jx); free(s->Jy); free(s->Hz);
    free(s->pexy); free(s->peyx); free(s->phzx); free(s->phzy);
}

/* Material of every edge: background eps_s; gap edges eps_g; design edges
 * Eq. (5a-c) of their own density (no filter in this mode). */
static void mat2t_build(const or_config *c, const double *rho, double sigma_max, double gamma_scale, mat2t *m)
{
    int nx = c->nx, ny = c->ny;
    size_t n = (size_t)nx * ny;
    m->gam = c->gamma_p * gamma_scale;
    for (int comp = 0; comp < 2; ++comp) {
        m->eps[comp] = malloc(n * sizeof(double));
        m->psi[comp] = calloc(n, sizeof(double));
        m->sig[comp] = calloc(n, sizeof(double));
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t q = (size_t)j * nx + i;
                m->eps[comp][q] = c->eps_s;
                long d = edge_index(c->design_lo, c->design_hi, comp, i, j);
                if (edge_index(c->gap_lo, c->gap_hi, comp, i, j) >= 0)
                    m->eps[comp][q] = c->eps_g;
                else if (d >= 0)
                    or_material(c, rho[d], sigma_max, &m->eps[comp][q], &m->psi[comp][q], &m->sig[comp][q]);
            }
    }
    m->ex = malloc(nx * sizeof(pml_coef)); m->hx = malloc(nx * sizeof(pml_coef));
    m->ey = malloc(ny * sizeof(pml_coef)); m->hy = malloc(ny * sizeof(pml_coef));
    or_config cx = *c;
    if (c->periodic_x) cx.npml = 0;
    for (int i = 0; i < nx; ++i) { m->ex[i] = pml_at(&cx, nx, i); m->hx[i] = pml_at(&cx, nx, i + 0.5); }
    for (int j = 0; j < ny; ++j) { m->ey[j] = pml_at(c, ny, j); m->hy[j] = pml_at(c, ny, j + 0.5); }
}

static void mat2t_free(mat2t *m)
{
    for (int comp = 0; comp < 2; ++comp) { free(m->eps[comp]); free(m->psi[comp]); free(m->sig[comp]); }
    free(m->ex); free(m->ey); free(m->hx); free(m->hy);
}

/* H half step: mu0 dHz/dt = -(dEy/dx - dEx/dy), forward differences. */
static void step2t_h(const or_config *c, const mat2t *m, st2t *s)
{
    int nx = c->nx, ny = c->ny, per = c->periodic_x;
    double dx = c->dx, ch = or_dt(c) / OR_MU0;
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < ny - 1; ++j)
        for (int i = 0; i < nx; ++i) {
            int ip = i + 1;
            if (ip == nx) {
                if (!per) continue;
                ip = 0;
            }
            size_t q = (size_t)j * nx + i;
            double dEy = (s->Ey[(size_t)j * nx + ip] - s->Ey[q]) / dx;
            double dEx = (s->Ex[q + nx] - s->Ex[q]) / dx;
            s->phzx[q] = m->hx[i].b * s->phzx[q] + m->hx[i].c * dEy;
            s->phzy[q] = m->hy[j].b * s->phzy[q] + m->hy[j].c * dEx;
            s->Hz[q] -= ch * (dEy / m->hx[i].kappa + s->phzx[q] - dEx / m->hy[j].kappa - s->phzy[q]);
        }
}

/* E, J half step: Eq. (10a,b) on every updated edge, with
 * curl_x = dHz/dy, curl_y = -dHz/dx (backward differences); jx, jy are the
 * source current densities per edge. */
static void step2t_e(const or_config *c, const mat2t *m, st2t *s, const double *jx, const double *jy)
{
    int nx = c->nx, ny = c->ny, per = c->periodic_x;
    double dt = or_dt(c), dx = c->dx;
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t q = (size_t)j * nx + i;
            /* Ex(i, j): an edge inside the grid, not on the rows j = 0, ny-1 */
            if (j >= 1 && j <= ny - 2 && (per || i <= nx - 2)) {
                double d = (s->Hz[q] - s->Hz[q - nx]) / dx;
                s->pexy[q] = m->ey[j].b * s->pexy[q] + m->ey[j].c * d;
                double curl = d / m->ey[j].kappa + s->pexy[q];
                node_solve(m->eps[0][q], m->psi[0][q], m->sig[0][q], m->gam, dt, curl, jx[q], &s->Ex[q], &s->Jx[q]);
            }
            /* Ey(i, j): not on the columns i = 0, nx-1 (unless periodic) */
            if (j <= ny - 2 && (per || (i >= 1 && i <= nx - 2))) {
                int im = i == 0 ? nx - 1 : i - 1;
                double d = (s->Hz[q] - s->Hz[(size_t)j * nx + im]) / dx;
                s->peyx[q] = m->ex[i].b * s->peyx[q] + m->ex[i].c * d;
                double curl = -(d / m->ex[i].kappa + s->peyx[q]);
                node_solve(m->eps[1][q], m->psi[1][q], m->sig[1][q], m->gam, dt, curl, jy[q], &s->Ey[q], &s->Jy[q]);
            }
        }
}

static double energy2t(const or_config *c, const mat2t *m, const st2t *s, const double *Hz_old)
{
    double eps0 = or_eps0(), e = 0.0;
    size_t n = (size_t)c->nx * c->ny;
    for (size_t q = 0; q < n; ++q) {
        e += 0.5 * eps0 * (m->eps[0][q] * s->Ex[q] * s->Ex[q] + m->eps[1][q] * s->Ey[q] * s->Ey[q]);
        e += 0.5 * OR_MU0 * Hz_old[q] * s->Hz[q];
    }
    return e * c->dx * c->dx;
}

/* Record the edges of a cell box (E_x edges, then E_y edges) of E^t. */
static void record_edges(const or_config *c, const int *lo, const int *hi, const st2t *s, double *out)
{
    int nx = c->nx;
    for (int comp = 0; comp < 2; ++comp) {
        const double *E = comp ? s->Ey : s->Ex;
        for (int j = lo[1]; j <= hi[1]; ++j)
            for (int i = lo[0]; i <= hi[0]; ++i) {
                long d = edge_index(lo, hi, comp, i, j);
                if (d >= 0) out[d] = E[(size_t)j * nx + i];
            }
    }
}

/* Forward solve, E in plane.  The source drives E_x edges of the source box
 * (i in [src_lo_x, src_hi_x), j in [src_lo_y, src_hi_y)); probes are E_x
 * edges (i, j). */
static int forward2t(const or_config *c, const double *rho, double sigma_max, double gamma_scale,
                     double *W, double *gap_hist, double *design_hist,
                     const int *probes, int nprobe, double *probe_hist, double *energy)
{
    int nx = c->nx, N = c->nsteps;
    long M, G;
    or_sizes(c, &M, &G);
    mat2t m;
    mat2t_build(c, rho, sigma_max, gamma_scale, &m);
    st2t s;
    st2t_alloc(c, &s);
    size_t n = (size_t)nx * c->ny;
    double *jx = calloc(n, sizeof(double)), *jy = calloc(n, sizeof(double));
    double *hzo = energy ? calloc(n, sizeof(double)) : NULL;
    double *gbuf = malloc(sizeof(double) * (G ? G : 1));
    double dt = or_dt(c);
    double J0 = c->src_amp * or_eps0() * OR_C0 / c->dx;
    double sum = 0.0;
    for (int t = 0; t <= N; ++t) {
        record_edges(c, c->gap_lo, c->gap_hi, &s, gbuf);
        for (long g = 0; g < G; ++g) sum += gbuf[g] * gbuf[g];
        if (gap_hist) memcpy(gap_hist + (size_t)t * G, gbuf, sizeof(double) * G);
        if (design_hist) record_edges(c, c->design_lo, c->design_hi, &s, design_hist + (size_t)t * M);
        for (int p = 0; p < nprobe; ++p)
            probe_hist[(size_t)t * nprobe + p] = s.Ex[(size_t)probes[2 * p + 1] * nx + probes[2 * p]];
        if (t == N) break;
        double js = J0 * or_signal(c, (t + 0.5) * dt);
        for (int j = c->src_lo[1]; j < c->src_hi[1]; ++j)
            for (int i = c->src_lo[0]; i < c->src_hi[0]; ++i)
                jx[(size_t)j * nx + i] = js;
        if (energy) memcpy(hzo, s.Hz, n * sizeof(double));
        step2t_h(c, &m, &s);
        if (energy) energy[t] = energy2t(c, &m, &s, hzo);
        step2t_e(c, &m, &s, jx, jy);
    }
    *W = 0.5 * c->eps_g * dt * c->dx * c->dx * sum;
    free(jx); free(jy); free(hzo); free(gbuf);
    st2t_free(&s);
    mat2t_free(&m);
    return 0;
}

/* Forward, adjoint and gradient, E in plane: the adjoint is the same solver
 * driven by J_src = -eps_g E^{N-n} on every gap edge (Eq. 20), and the
 * Eq. (25a-c) sums run over every design edge with that edge's own forward
 * field, adjoint field and current, then Eq. (27) per edge (no filter);
 * gap edges get a zero gradient. */
static int gradient2t(const or_config *c, const double *rho, double sigma_max, double gamma_scale,
                      double *W, double *grad, double *g_psi, double *g_eps, double *g_sig)
{
    int nx = c->nx, N = c->nsteps;
    long M, G;
    or_sizes(c, &M, &G);
    if (M == 0) return -1;
    double *ghist = malloc(sizeof(double) * (size_t)(N + 1) * (G ? G : 1));
    double *dhist = malloc(sizeof(double) * (size_t)(N + 1) * M);
    forward2t(c, rho, sigma_max, gamma_scale, W, ghist, dhist, NULL, 0, NULL, NULL);
    mat2t m;
    mat2t_build(c, rho, sigma_max, gamma_scale, &m);
    st2t a;
    st2t_alloc(c, &a);
    size_t n = (size_t)nx * c->ny;
    double *jx = calloc(n, sizeof(double)), *jy = calloc(n, sizeof(double));
    double *sp = calloc(M, sizeof(double)), *se = calloc(M, sizeof(double)), *ss = calloc(M, sizeof(double));
    double *Eold = malloc(sizeof(double) * M), *Jold = malloc(sizeof(double) * M);
    double *Enew = malloc(sizeof(double) * M), *Jnew = malloc(sizeof(double) * M);
    st2t jview = a;
    for (int t = 0; t <= N; ++t) {
        for (int comp = 0; comp < 2; ++comp)
            for (int j = c->gap_lo[1]; j <= c->gap_hi[1]; ++j)
                for (int i = c->gap_lo[0]; i <= c->gap_hi[0]; ++i) {
                    long g = edge_index(c->gap_lo, c->gap_hi, comp, i, j);
                    if (g >= 0) (comp ? jy : jx)[(size_t)j * nx + i] = -c->eps_g * ghist[(size_t)(N - t) * G + g];
                }
        record_edges(c, c->design_lo, c->design_hi, &a, Eold);
        jview.Ex = a.Jx;
        jview.Ey = a.Jy;
        record_edges(c, c->design_lo, c->design_hi, &jview, Jold);
        step2t_h(c, &m, &a);
        step2t_e(c, &m, &a, jx, jy);
        record_edges(c, c->design_lo, c->design_hi, &a, Enew);
        record_edges(c, c->design_lo, c->design_hi, &jview, Jnew);
        for (long d = 0; d < M; ++d) {
            double Ef = dhist[(size_t)(N - t) * M + d];
            sp[d] += Ef * 0.5 * (Jnew[d] + Jold[d]);
            se[d] += Ef * (Enew[d] - Eold[d]);
            ss[d] += Ef * 0.5 * (Enew[d] + Eold[d]);
        }
    }
    double eps0 = or_eps0(), dt = or_dt(c), dx2 = c->dx * c->dx;
    double psi = c->omega_p * c->omega_p, psi_s = c->psi_s_ratio * psi;
    for (int comp = 0; comp < 2; ++comp)
        for (int j = c->design_lo[1]; j <= c->design_hi[1]; ++j)
            for (int i = c->design_lo[0]; i <= c->design_hi[0]; ++i) {
                long d = edge_index(c->design_lo, c->design_hi, comp, i, j);
                if (d < 0) continue;
                double ep, ps, sg;
                or_material(c, rho[d], sigma_max, &ep, &ps, &sg);
                double dpsi = -(dt * dx2 / ps) * sp[d];
                double deps = -eps0 * dx2 * se[d];
                double dsig = -dt * dx2 * ss[d];
                if (edge_index(c->gap_lo, c->gap_hi, comp, i, j) >= 0) dpsi = deps = dsig = 0.0;
                if (g_psi) g_psi[d] = dpsi;
                if (g_eps) g_eps[d] = deps;
                if (g_sig) g_sig[d] = dsig;
                double dsdr = sigma_max * (1.0 - 2.0 * rho[d]) * (c->sigma_form ? 4.0 : 1.0);
                grad[d] = (psi - psi_s) * dpsi + (c->eps_inf - c->eps_s) * deps + dsdr * dsig;
            }
    free(Eold); free(Jold); free(Enew); free(Jnew); free(sp); free(se); free(ss);
    free(jx); free(jy); free(ghist); free(dhist);
    st2t_free(&a);
    mat2t_free(&m);
    return 0;
}

/* ================================================================ 3D */

/* Full Yee grid of nx x ny x nz nodes: Ex(i,j,k) at (i+1/2, j, k), Ey at
 * (i, j+1/2, k), Ez at (i, j, k+1/2), Hx at (i, j+1/2, k+1/2), Hy at
 * (i+1/2, j, k+1/2), Hz at (i+1/2, j+1/2, k).  Tangential E vanishes on the
 * outer faces (PEC walls behind the CPML).  Every component of index
 * (i, j, k) in the design box takes the material of rho(i, j, k); J is kept
 * per E component.  All arrays are whole [nz][ny][nx]. */

enum { X = 0, Y = 1, Z = 2 };

typedef struct {
    double *E[3], *J[3], *H[3];
    double *pe[3][3], *ph[3][3];   /* CPML term of component c along axis a */
} st3;

typedef struct {
    double *eps[3], *psi[3], *sig[3];  /* per E component */
    double gam;
    pml_coef *e[3], *h[3];             /* per axis, at node / half positions */
} mat3;

static size_t n3(const or_config *c) { return (size_t)c->nx * c->ny * c->nz; }
static size_t id3(const or_config *c, int i, int j, int k) { return ((size_t)k * c->ny + j) * c->nx + i; }

static void st3_alloc(const or_config *c, st3 *s)
{
    size_t n = n3(c);
    for (int a = 0; a < 3; ++a) {
        s->E[a] = calloc(n, sizeof(double));
        s->J[a] = calloc(n, sizeof(double));
        s->H[a] = calloc(n, sizeof(double));
        for (int b = 0; b < 3; ++b) {
            s->pe[a][b] = calloc(n, sizeof(double));
            s->ph[a][b] = calloc(n, sizeof(double));
        }
    }
}

static void st3_free(st3 *s)
{
    for (int a = 0; a < 3; ++a) {
        free(s->E[a]); free(s->J[a]); free(s->H[a]);
        for (int b = 0; b < 3; ++b) { free(s->pe[a][b]); free(s->ph[a][b]); }
    }
}

static void mat3_build(const or_config *c, const double *rho_t, double sigma_max, double gamma_scale, mat3 *m)
{
    size_t n = n3(c);
    int dw = c->design_hi[0] - c->design_lo[0], dh = c->design_hi[1] - c->design_lo[1];
    m->gam = c->gamma_p * gamma_scale;
    for (int a = 0; a < 3; ++a) {
        m->eps[a] = malloc(n * sizeof(double));
        m->psi[a] = calloc(n, sizeof(double));
        m->sig[a] = calloc(n, sizeof(double));
    }
    for (int k = 0; k < c->nz; ++k)
        for (int j = 0; j < c->ny; ++j)
            for (int i = 0; i < c->nx; ++i) {
                size_t q = id3(c, i, j, k);
                double eb = k < c->sub_hi ? c->sub_eps : c->eps_s;
                double e = eb, p = 0.0, sg = 0.0;
                if (in_box(c->gap_lo, c->gap_hi, i, j, k)) {
                    e = c->eps_g;
                } else if (in_box(c->design_lo, c->design_hi, i, j, k)) {
                    double r = rho_t[((size_t)(k - c->design_lo[2]) * dh + (j - c->design_lo[1])) * dw +
                                     (i - c->design_lo[0])];
                    or_material(c, r, sigma_max, &e, &p, &sg);
                }
                for (int a = 0; a < 3; ++a) { m->eps[a][q] = e; m->psi[a][q] = p; m->sig[a][q] = sg; }
            }
    int nn[3] = {c->nx, c->ny, c->nz};
    for (int a = 0; a < 3; ++a) {
        m->e[a] = malloc(nn[a] * sizeof(pml_coef));
        m->h[a] = malloc(nn[a] * sizeof(pml_coef));
        for (int i = 0; i < nn[a]; ++i) {
            m->e[a][i] = pml_at(c, nn[a], i);
            m->h[a][i] = pml_at(c, nn[a], i + 0.5);
        }
    }
}

static void mat3_free(mat3 *m)
{
    for (int a = 0; a < 3; ++a) {
        free(m->eps[a]); free(m->psi[a]); free(m->sig[a]); free(m->e[a]); free(m->h[a]);
    }
}

/* d/d(axis) of field F at node (i, j, k), forward difference (for H from E)
 * or backward difference (for E from H), divided by dx; 0 where the
 * neighbour is outside the grid. */
static double dfwd(const or_config *c, const double *F, int ax, int i, int j, int k)
{
    int ii = i + (ax == X), jj = j + (ax == Y), kk = k + (ax == Z);
    if (ii >= c->nx || jj >= c->ny || kk >= c->nz) return 0.0;
    return (F[id3(c, ii, jj, kk)] - F[id3(c, i, j, k)]) / c->dx;
}

static double dbwd(const or_config *c, const double *F, int ax, int i, int j, int k)
{
    int ii = i - (ax == X), jj = j - (ax == Y), kk = k - (ax == Z);
    if (ii < 0 || jj < 0 || kk < 0) return 0.0;
    return (F[id3(c, i, j, k)] - F[id3(c, ii, jj, kk)]) / c->dx;
}

/* Is component comp of E (or H) at index (i, j, k) inside the grid and, for
 * E, away from the PEC walls (tangential E = 0 on the outer faces)? */
static int e_active(const or_config *c, int comp, int i, int j, int k)
{
    int n[3] = {c->nx, c->ny, c->nz}, p[3] = {i, j, k};
    for (int a = 0; a < 3; ++a) {
        if (a == comp) { if (p[a] > n[a] - 2) return 0; }
        else if (p[a] < 1 || p[a] > n[a] - 2) return 0;
    }
    return 1;
}

static int h_active(const or_config *c, int comp, int i, int j, int k)
{
    int n[3] = {c->nx, c->ny, c->nz}, p[3] = {i, j, k};
    for (int a = 0; a < 3; ++a)
        if (a != comp && p[a] > n[a] - 2) return 0;
    return 1;
}

/* The two (axis, sign) terms of curl component comp: curl_c = d_a F_b - d_b F_a
 * with (c, a, b) cyclic. */
static void curl_axes(int comp, int *a, int *b) { *a = (comp + 1) % 3; *b = (comp + 2) % 3; }

/* ------------------------------------------- plane wave by TFSF (3D) */

/* The incident wave is x-polarised and travels along +z.  It is the field
 * of the laterally uniform problem: a 1D Yee column along z with the 3D
 * grid's background layering (sub_eps below sub_hi, eps_s above), its
 * z-CPML and PEC ends, driven by the soft E_x current of the source plane
 * k = src_lo[2].  In the column E_x(k) sits at z = k and H_y(k) at
 * z = k + 1/2, exactly where the 3D components of the same index sit, and
 * each update is the 3D one with the x and y derivatives zero.
 *
 * The 3D arrays hold the total field at every component whose Yee position
 * lies in the closed box tf_lo <= x <= tf_hi, and the scattered field
 * elsewhere.  A difference taken at a field F that reaches a sample of a
 * field G across the box boundary converts the sample into F's view first:
 * G + (tf(F) - tf(G)) G_inc. */
typedef struct {
    int nz;
    double *E, *H, *pe, *ph;     /* E_x, H_y and their z-CPML terms */
    pml_coef *ce, *ch;           /* z-CPML at nodes / half positions */
    double *eps;                 /* background permittivity per k */
    double gam;
} col1d;

static void col_init(const or_config *c, double gamma_scale, col1d *L)
{
    int nz = c->nz;
    L->nz = nz;
    L->E = calloc(nz, sizeof(double)); L->H = calloc(nz, sizeof(double));
    L->pe = calloc(nz, sizeof(double)); L->ph = calloc(nz, sizeof(double));
    L->ce = malloc(nz * sizeof(pml_coef)); L->ch = malloc(nz * sizeof(pml_coef));
    L->eps = malloc(nz * sizeof(double));
    for (int k = 0; k < nz; ++k) {
        L->ce[k] = pml_at(c, nz, k);
        L->ch[k] = pml_at(c, nz, k + 0.5);
        L->eps[k] = k < c->sub_hi ? c->sub_eps : c->eps_s;
    }
    L->gam = c->gamma_p * gamma_scale;
}

static void col_free(col1d *L)
{
    free(L->E); free(L->H); free(L->pe); free(L->ph); free(L->ce); free(L->ch); free(L->eps);
}

/* mu0 dH_y/dt = -(dE_x/dz), the y row of the 3D H update. */
static void col_h(const or_config *c, col1d *L)
{
    double ch = or_dt(c) / OR_MU0;
    for (int k = 0; k + 1 < L->nz; ++k) {
        double d = (L->E[k + 1] - L->E[k]) / c->dx;
        pml_coef p = L->ch[k];
        L->ph[k] = p.b * L->ph[k] + p.c * d;
        L->H[k] -= ch * (d / p.kappa + L->ph[k]);
    }
}

/* E_x from curl_x H = -dH_y/dz and the source current jsrc on its plane. */
static void col_e(const or_config *c, col1d *L, double jsrc)
{
    for (int k = 1; k + 1 < L->nz; ++k) {
        double d = (L->H[k] - L->H[k - 1]) / c->dx;
        pml_coef p = L->ce[k];
        L->pe[k] = p.b * L->pe[k] + p.c * d;
        double curl = -(d / p.kappa + L->pe[k]);
        double J = 0.0;
        node_solve(L->eps[k], 0.0, 0.0, L->gam, or_dt(c), curl,
                   (k >= c->src_lo[2] && k < c->src_hi[2]) ? jsrc : 0.0, &L->E[k], &J);
    }
}

/* Is component comp of E (isH = 0) or H (isH = 1) of index (i, j, k) in the
 * total-field box?  E_c sits half a cell along c, H_c half a cell along the
 * other two axes. */
static int tf_in(const or_config *c, int isH, int comp, int i, int j, int k)
{
    int p[3] = {i, j, k};
    for (int a = 0; a < 3; ++a) {
        double x = p[a] + (((a == comp) != isH) ? 0.5 : 0.0);
        if (x < c->tf_lo[a] || x > c->tf_hi[a]) return 0;
    }
    return 1;
}

/* Incident value of a component: only E_x and H_y are non-zero. */
static double inc_at(const col1d *L, int isH, int comp, int k)
{
    if (!isH) return comp == X ? L->E[k] : 0.0;
    return comp == Y ? L->H[k] : 0.0;
}

/* (tf(F) - tf(G)) G_inc for the sample of G (kind isH, component comp) at
 * (i, j, k), seen from a field F whose flag is tfF. */
static double tf_shift(const or_config *c, const col1d *L, int tfF, int isH, int comp, int i, int j, int k)
{
    int d = tfF - tf_in(c, isH, comp, i, j, k);
    return d ? d * inc_at(L, isH, comp, k) : 0.0;
}

/* H half step: mu0 dH/dt = -curl E with CPML on each derivative; with a
 * column L, the E samples are converted as described above. */
static void step3_h(const or_config *c, const mat3 *m, st3 *s, const col1d *L)
{
    double ch = or_dt(c) / OR_MU0;
    #pragma omp parallel for schedule(static)
    for (int k = 0; k < c->nz; ++k)
        for (int j = 0; j < c->ny; ++j)
            for (int i = 0; i < c->nx; ++i) {
                int p[3] = {i, j, k};
                size_t q = id3(c, i, j, k);
                for (int comp = 0; comp < 3; ++comp) {
                    if (!h_active(c, comp, i, j, k)) continue;
                    int a, b;
                    curl_axes(comp, &a, &b);
                    /* curl_comp E = d_a E_b - d_b E_a */
                    double da = dfwd(c, s->E[b], a, i, j, k);
                    double db = dfwd(c, s->E[a], b, i, j, k);
                    if (L) {
                        int tfF = tf_in(c, 1, comp, i, j, k);
                        int ea[3] = {a == X, a == Y, a == Z}, eb[3] = {b == X, b == Y, b == Z};
                        if (p[a] + 1 < (a == X ? c->nx : a == Y ? c->ny : c->nz))
                            da += (tf_shift(c, L, tfF, 0, b, i + ea[0], j + ea[1], k + ea[2]) -
                                   tf_shift(c, L, tfF, 0, b, i, j, k)) / c->dx;
                        if (p[b] + 1 < (b == X ? c->nx : b == Y ? c->ny : c->nz))
                            db += (tf_shift(c, L, tfF, 0, a, i + eb[0], j + eb[1], k + eb[2]) -
                                   tf_shift(c, L, tfF, 0, a, i, j, k)) / c->dx;
                    }
                    pml_coef pa = m->h[a][p[a]], pb = m->h[b][p[b]];
                    s->ph[comp][a][q] = pa.b * s->ph[comp][a][q] + pa.c * da;
                    s->ph[comp][b][q] = pb.b * s->ph[comp][b][q] + pb.c * db;
                    double curl = da / pa.kappa + s->ph[comp][a][q] - db / pb.kappa - s->ph[comp][b][q];
                    s->H[comp][q] -= ch * curl;
                }
            }
}

/* E, J half step: Eq. (10a,b) for every active E component; jsrc[comp] is a
 * per-node current density (or NULL); with a column L, the H samples are
 * converted as described above. */
static void step3_e(const or_config *c, const mat3 *m, st3 *s, double *const *jsrc, const col1d *L)
{
    double dt = or_dt(c);
    #pragma omp parallel for schedule(static)
    for (int k = 0; k < c->nz; ++k)
        for (int j = 0; j < c->ny; ++j)
            for (int i = 0; i < c->nx; ++i) {
                int p[3] = {i, j, k};
                size_t q = id3(c, i, j, k);
                for (int comp = 0; comp < 3; ++comp) {
                    if (!e_active(c, comp, i, j, k)) continue;
                    int a, b;
                    curl_axes(comp, &a, &b);
                    double da = dbwd(c, s->H[b], a, i, j, k);
                    double db = dbwd(c, s->H[a], b, i, j, k);
                    if (L) {
                        int tfF = tf_in(c, 0, comp, i, j, k);
                        int ea[3] = {a == X, a == Y, a == Z}, eb[3] = {b == X, b == Y, b == Z};
                        if (p[a] >= 1)
                            da += (tf_shift(c, L, tfF, 1, b, i, j, k) -
                                   tf_shift(c, L, tfF, 1, b, i - ea[0], j - ea[1], k - ea[2])) / c->dx;
                        if (p[b] >= 1)
                            db += (tf_shift(c, L, tfF, 1, a, i, j, k) -
                                   tf_shift(c, L, tfF, 1, a, i - eb[0], j - eb[1], k - eb[2])) / c->dx;
                    }
                    pml_coef pa = m->e[a][p[a]], pb = m->e[b][p[b]];
                    s->pe[comp][a][q] = pa.b * s->pe[comp][a][q] + pa.c * da;
                    s->pe[comp][b][q] = pb.b * s->pe[comp][b][q] + pb.c * db;
                    double curl = da / pa.kappa + s->pe[comp][a][q] - db / pb.kappa - s->pe[comp][b][q];
                    node_solve(m->eps[comp][q], m->psi[comp][q], m->sig[comp][q], m->gam, dt, curl,
                               jsrc && jsrc[comp] ? jsrc[comp][q] : 0.0, &s->E[comp][q], &s->J[comp][q]);
                }
            }
}

static double energy3(const or_config *c, const mat3 *m, const st3 *s, double *const *Hold)
{
    double eps0 = or_eps0(), e = 0.0;
    size_t n = n3(c);
    for (int a = 0; a < 3; ++a)
        for (size_t q = 0; q < n; ++q) {
            e += 0.5 * eps0 * m->eps[a][q] * s->E[a][q] * s->E[a][q];
            e += 0.5 * OR_MU0 * Hold[a][q] * s->H[a][q];
        }
    return e * c->dx * c->dx * c->dx;
}

/* Gap / design boxes hold 3 components per index: history layout
 * [t][comp][box index]. */
static int forward3(const or_config *c, const double *rho, double sigma_max, double gamma_scale, double *W,
                    double *gap_hist, double *design_hist, const int *probes, int nprobe, double *probe_hist,
                    double *energy)
{
    int N = c->nsteps;
    long M, G;
    or_sizes(c, &M, &G);
    double *rho_t = malloc(sizeof(double) * (M ? M : 1));
    if (M) or_filter(c, rho, rho_t);
    mat3 m;
    mat3_build(c, rho_t, sigma_max, gamma_scale, &m);
    st3 s;
    st3_alloc(c, &s);
    size_t n = n3(c);
    double *js[3] = {NULL, NULL, NULL};
    js[c->src_comp] = calloc(n, sizeof(double));
    const int tf = c->tfsf != 0;
    col1d col;
    if (tf) col_init(c, gamma_scale, &col);
    double *Hold[3] = {NULL, NULL, NULL};
    if (energy)
        for (int a = 0; a < 3; ++a) Hold[a] = calloc(n, sizeof(double));
    double dt = or_dt(c);
    double J0 = c->src_amp * or_eps0() * OR_C0 / c->dx;
    double sum = 0.0;
    int gw = c->gap_hi[0] - c->gap_lo[0], gh = c->gap_hi[1] - c->gap_lo[1];
    int dw = c->design_hi[0] - c->design_lo[0], dh = c->design_hi[1] - c->design_lo[1];
    for (int t = 0; t <= N; ++t) {
        for (int a = 0; a < 3; ++a) {
            for (int k = c->gap_lo[2]; k < c->gap_hi[2]; ++k)
                for (int j = c->gap_lo[1]; j < c->gap_hi[1]; ++j)
                    for (int i = c->gap_lo[0]; i < c->gap_hi[0]; ++i) {
                        double e = s.E[a][id3(c, i, j, k)];
                        sum += e * e;
                        if (gap_hist)
                            gap_hist[((size_t)t * 3 + a) * G +
                                     ((size_t)(k - c->gap_lo[2]) * gh + (j - c->gap_lo[1])) * gw + (i - c->gap_lo[0])] = e;
                    }
            if (design_hist)
                for (int k = c->design_lo[2]; k < c->design_hi[2]; ++k)
                    for (int j = c->design_lo[1]; j < c->design_hi[1]; ++j)
                        for (int i = c->design_lo[0]; i < c->design_hi[0]; ++i)
                            design_hist[((size_t)t * 3 + a) * M +
                                        ((size_t)(k - c->design_lo[2]) * dh + (j - c->design_lo[1])) * dw +
                                        (i - c->design_lo[0])] = s.E[a][id3(c, i, j, k)];
        }
        for (int pi = 0; pi < nprobe; ++pi)
            probe_hist[(size_t)t * nprobe + pi] =
                s.E[probes[4 * pi + 3]][id3(c, probes[4 * pi], probes[4 * pi + 1], probes[4 * pi + 2])];
        if (t == N) break;
        double v = J0 * or_signal(c, (t + 0.5) * dt);
        if (!tf)
            for (int k = c->src_lo[2]; k < c->src_hi[2]; ++k)
                for (int j = c->src_lo[1]; j < c->src_hi[1]; ++j)
                    for (int i = c->src_lo[0]; i < c->src_hi[0]; ++i) js[c->src_comp][id3(c, i, j, k)] = v;
        if (energy)
            for (int a = 0; a < 3; ++a) memcpy(Hold[a], s.H[a], n * sizeof(double));
        /* 3D H from E^t (incident E^t), then the column's H^{t+1/2}; 3D E
         * from H^{t+1/2}, then the column's E^{t+1} */
        step3_h(c, &m, &s, tf ? &col : NULL);
        if (tf) col_h(c, &col);
        if (energy) energy[t] = energy3(c, &m, &s, Hold);
        step3_e(c, &m, &s, js, tf ? &col : NULL);
        if (tf) col_e(c, &col, v);
    }
    if (tf) col_free(&col);
    *W = 0.5 * c->eps_g * dt * c->dx * c->dx * c->dx * sum;
    free(js[c->src_comp]);
    for (int a = 0; a < 3; ++a) free(Hold[a]);
    free(rho_t);
    st3_free(&s);
    mat3_free(&m);
    return 0;
}

/* Adjoint (Eq. 20) and sensitivities (Eq. 25) per E component, summed over
 * the three components of each design index, then Eq. (27). */
static int gradient3(const or_config *c, const double *rho, double sigma_max, double gamma_scale, double *W,
                     double *grad, double *g_psi, double *g_eps, double *g_sig)
{
    int N = c->nsteps;
    long M, G;
    or_sizes(c, &M, &G);
    if (M == 0) return -1;
    double *ghist = malloc(sizeof(double) * (size_t)(N + 1) * 3 * (G ? G : 1));
    double *dhist = malloc(sizeof(double) * (size_t)(N + 1) * 3 * M);
    forward3(c, rho, sigma_max, gamma_scale, W, ghist, dhist, NULL, 0, NULL, NULL);
    double *rho_t = malloc(sizeof(double) * M);
    or_filter(c, rho, rho_t);
    mat3 m;
    mat3_build(c, rho_t, sigma_max, gamma_scale, &m);
    st3 s;
    st3_alloc(c, &s);
    size_t n = n3(c);
    double *js[3];
    for (int a = 0; a < 3; ++a) js[a] = calloc(n, sizeof(double));
    double *sp = calloc(M, sizeof(double)), *se = calloc(M, sizeof(double)), *ss = calloc(M, sizeof(double));
    double *Eo = malloc(sizeof(double) * 3 * M), *Jo = malloc(sizeof(double) * 3 * M);
    int gw = c->gap_hi[0] - c->gap_lo[0], gh = c->gap_hi[1] - c->gap_lo[1];
    int dw = c->design_hi[0] - c->design_lo[0], dh = c->design_hi[1] - c->design_lo[1];
    for (int t = 0; t <= N; ++t) {
        for (int a = 0; a < 3; ++a)
            for (int k = c->gap_lo[2]; k < c->gap_hi[2]; ++k)
                for (int j = c->gap_lo[1]; j < c->gap_hi[1]; ++j)
                    for (int i = c->gap_lo[0]; i < c->gap_hi[0]; ++i)
                        js[a][id3(c, i, j, k)] =
                            -c->eps_g * ghist[((size_t)(N - t) * 3 + a) * G +
                                              ((size_t)(k - c->gap_lo[2]) * gh + (j - c->gap_lo[1])) * gw +
                                              (i - c->gap_lo[0])];
        for (int a = 0; a < 3; ++a)
            for (int k = c->design_lo[2]; k < c->design_hi[2]; ++k)
                for (int j = c->design_lo[1]; j < c->design_hi[1]; ++j)
                    for (int i = c->design_lo[0]; i < c->design_hi[0]; ++i) {
                        long d = ((long)(k - c->design_lo[2]) * dh + (j - c->design_lo[1])) * dw + (i - c->design_lo[0]);
                        Eo[a * M + d] = s.E[a][id3(c, i, j, k)];
                        Jo[a * M + d] = s.J[a][id3(c, i, j, k)];
                    }
        step3_h(c, &m, &s, NULL);
        step3_e(c, &m, &s, js, NULL);
        for (int a = 0; a < 3; ++a)
            for (int k = c->design_lo[2]; k < c->design_hi[2]; ++k)
                for (int j = c->design_lo[1]; j < c->design_hi[1]; ++j)
                    for (int i = c->design_lo[0]; i < c->design_hi[0]; ++i) {
                        long d = ((long)(k - c->design_lo[2]) * dh + (j - c->design_lo[1])) * dw + (i - c->design_lo[0]);
                        size_t q = id3(c, i, j, k);
                        double Ef = dhist[((size_t)(N - t) * 3 + a) * M + d];
                        sp[d] += Ef * 0.5 * (s.J[a][q] + Jo[a * M + d]);
                        se[d] += Ef * (s.E[a][q] - Eo[a * M + d]);
                        ss[d] += Ef * 0.5 * (s.E[a][q] + Eo[a * M + d]);
                    }
    }
    double eps0 = or_eps0(), dt = or_dt(c), dx3 = c->dx * c->dx * c->dx;
    double psi = c->omega_p * c->omega_p, psi_s = c->psi_s_ratio * psi;
    double *gt = malloc(sizeof(double) * M);
    for (int k = c->design_lo[2]; k < c->design_hi[2]; ++k)
        for (int j = c->design_lo[1]; j < c->design_hi[1]; ++j)
            for (int i = c->design_lo[0]; i < c->design_hi[0]; ++i) {
                long d = ((long)(k - c->design_lo[2]) * dh + (j - c->design_lo[1])) * dw + (i - c->design_lo[0]);
                double ep, ps, sg;
                or_material(c, rho_t[d], sigma_max, &ep, &ps, &sg);
                double dpsi = -(dt * dx3 / ps) * sp[d];
                double deps = -eps0 * dx3 * se[d];
                double dsig = -dt * dx3 * ss[d];
                if (in_box(c->gap_lo, c->gap_hi, i, j, k)) dpsi = deps = dsig = 0.0;
                if (g_psi) g_psi[d] = dpsi;
                if (g_eps) g_eps[d] = deps;
                if (g_sig) g_sig[d] = dsig;
                double dsdr = sigma_max * (1.0 - 2.0 * rho_t[d]) * (c->sigma_form ? 4.0 : 1.0);
                gt[d] = (psi - psi_s) * dpsi + (c->eps_inf - c->eps_s) * deps + dsdr * dsig;
            }
    or_filter_T(c, gt, grad);
    for (int k = c->gap_lo[2]; k < c->gap_hi[2]; ++k)
        for (int j = c->gap_lo[1]; j < c->gap_hi[1]; ++j)
            for (int i = c->gap_lo[0]; i < c->gap_hi[0]; ++i)
                grad[((long)(k - c->design_lo[2]) * dh + (j - c->design_lo[1])) * dw + (i - c->design_lo[0])] = 0.0;
    free(gt); free(Eo); free(Jo); free(sp); free(se); free(ss);
    for (int a = 0; a < 3; ++a) free(js[a]);
    free(rho_t); free(ghist); free(dhist);
    st3_free(&s);
    mat3_free(&m);
    return 0;
}

/* ============================================================ public */

/* The incident plane wave of a 3D workload with tfsf = 1: E_x at nodes ks[]
 * for t = 0..N ((N+1) x nk, E_out) and H_y at the same indices for
 * t + 1/2, t = 0..N-1 (N x nk, H_out). */
int or_tfsf_incident(const or_config *c, double gamma_scale, const int *ks, int nk, double *E_out,
                     double *H_out)
{
    if (c->ndim != 3) return -1;
    col1d col;
    col_init(c, gamma_scale, &col);
    double dt = or_dt(c), J0 = c->src_amp * or_eps0() * OR_C0 / c->dx;
    for (int t = 0; t <= c->nsteps; ++t) {
        for (int q = 0; q < nk; ++q) E_out[(size_t)t * nk + q] = col.E[ks[q]];
        if (t == c->nsteps) break;
        col_h(c, &col);
        for (int q = 0; q < nk; ++q) H_out[(size_t)t * nk + q] = col.H[ks[q]];
        col_e(c, &col, J0 * or_signal(c, (t + 0.5) * dt));
    }
    col_free(&col);
    return 0;
}

int or_forward(const or_config *c, const double *rho, double sigma_max, double gamma_scale,
               double *W, double *gap_hist, double *design_hist,
               const int *probes, int nprobe, double *probe_hist, double *energy)
{
    if (c->ndim == 2 && c->pol == 1)
        return forward2t(c, rho, sigma_max, gamma_scale, W, gap_hist, design_hist,
                         probes, nprobe, probe_hist, energy);
    if (c->ndim == 2)
        return forward2(c, rho, sigma_max, gamma_scale, W, gap_hist, design_hist,
                        probes, nprobe, probe_hist, energy);
    if (c->ndim == 3)
        return forward3(c, rho, sigma_max, gamma_scale, W, gap_hist, design_hist,
                        probes, nprobe, probe_hist, energy);
    return -1;
}

int or_gradient(const or_config *c, const double *rho, double sigma_max, double gamma_scale,
                double *W, double *grad, double *g_psi, double *g_eps, double *g_sig)
{
    if (c->ndim == 2 && c->pol == 1) return gradient2t(c, rho, sigma_max, gamma_scale, W, grad, g_psi, g_eps, g_sig);
    if (c->ndim == 2) return gradient2(c, rho, sigma_max, gamma_scale, W, grad, g_psi, g_eps, g_sig);
    if (c->ndim == 3) return gradient3(c, rho, sigma_max, gamma_scale, W, grad, g_psi, g_eps, g_sig);
    return -1;
}
