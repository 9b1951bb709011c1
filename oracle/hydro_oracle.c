/*
 * hydro_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, FP64 CPU statement of one step of the unsplit finite-volume
 * update of the compressible Euler equations (gamma-law gas, constant
 * gravity): PLM reconstruction with the MC limiter, single-stage unsplit
 * MUSCL-Hancock half-step predictor in primitive variables, an HLLC flux at
 * every face, flux divergence plus gravity source, and the CFL time step.
 *
 * The paper ("Modeling Astrophysical Explosions with Sustained Exascale
 * Computing", introduction) describes a star modelled as a fluid on a
 * domain-decomposed grid, with nearest-neighbour plus global communication
 * every time step ("Capabilities needed").  It prints no scheme; every
 * numerical choice below is stated where it is made and credited to the
 * textbook or published method it follows:
 *   - unsplit single-stage MUSCL-Hancock (van Leer 1984; Toro, 3rd ed.,
 *     sec. 14.4) in primitive variables, all axes and half a step of gravity
 *     in the predictor; a cell whose predicted face density or pressure is
 *     not positive falls back to zero slopes;
 *   - HLLC with Davis wave speeds (Toro sec. 10.4-10.6), tie S* = 0 left;
 *   - gravity: momentum source g (rho^n + rho^{n+1})/2 with density updated
 *     first, energy source g . (mass flux through the low face + mass flux
 *     through the high face)/2;
 *   - dt = cfl / max_cells sum_d (|u_d| + c)/dx_d from the current state,
 *     the last step clamped to land on t_end; time accumulated in FP64;
 *   - boundaries by index mapping (outflow = clamp, periodic = wrap,
 *     reflecting = mirror with the normal momentum negated); at a reflecting
 *     wall the far-side face state is the mirror of the near side's.
 *
 * Second integrator (scheme = 1): the method of lines with the two-stage
 * strong-stability-preserving Runge-Kutta method of Shu and Osher (1988),
 *   U1 = U^n + dt L(U^n),   U^{n+1} = (U^n + U1 + dt L(U1)) / 2,
 * where L is the same spatial operator without the half-step predictor: face
 * states W -/+ dW/2 from the MC slopes (same positivity fallback), HLLC,
 * flux divergence, momentum source g rho of the stage state and the same
 * mass-flux energy source.  dt is taken from U^n.
 *
 * Third integrator (scheme = 2, PLM only): the unsplit corner
 * transport upwind method of Colella (1990): per axis d a one-dimensional
 * MUSCL-Hancock predictor (only the axis's own A_d term, half a step of
 * gravity) gives face states; HLLC fluxes from those states at every face
 * (first pass); each face state is corrected in conserved variables by the
 * transverse flux differences of its own cell, -dt/(2 dx_e) (F_e(+) -
 * F_e(-)) for every other axis e (kept uncorrected for a cell whose
 * corrected pair along d would have a non-positive density or pressure);
 * HLLC again on the corrected states; the update and sources of the
 * MUSCL-Hancock step.  In hydrostatic-background mode the scheme is the
 * plain one rewritten on perturbations: the z predictor advects the
 * background and takes g rho'/rho - B_k/rho (as the MUSCL-Hancock half step
 * does), the x and y predictors take g; a face state is corrected as a total
 * state (background at the face added before, removed after), and since the
 * first-pass z fluxes carry p', the background's pressure difference across
 * the cell is added to the z-momentum correction of x and y states.
 *
 * Second reconstruction (recon = 1, with scheme = 1 and hse = 0 only): the
 * piecewise parabolic method of Colella and Woodward (1984) in primitive
 * variables, used as the method of lines' face states: the interface value
 * a_{i+1/2} = (a_i + a_{i+1})/2 - (dm_{i+1} - dm_i)/6 from the MC-limited
 * slopes dm (their eqs. 1.7-1.9 on a uniform grid), then the parabola of
 * cell i limited to be monotone (their eq. 1.10).  Needs three ghost cells.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this file's library.  It shares no code with the CUDA path.
 *
 * Layout: a state is nvar planes U[q][k][j][i] (x fastest), conserved
 * variables (rho, rho u_0 .. rho u_{ndim-1}, E).  Internally every array is
 * padded by 2 ghost cells on each side of each active axis, ghosts are
 * filled explicitly, and primitives, slopes, face states and face fluxes
 * each live in their own array.  Compiled with -ffp-contract=off.
 *
 * Hydrostatic-background mode (hse = 1, 3D, gravity along z): the state is
 * the perturbation U' = U - U0(z), U0 = (rho0, 0, 0, 0, p0/(gamma-1)); the
 * reconstruction acts on (rho', u, p'), the background is added back at
 * faces from the given FP64 tables, and the momentum flux carries p' with
 * the background's discrete imbalance B_k applied as a source.  With zero
 * background tables every formula reduces exactly to the plain scheme, so
 * one code path serves both modes.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NG 2        /* ghost depth: PLM slope of a face-neighbour */
#define NG_PPM 3    /* PPM: interface values of a face-neighbour */
#define MAXV 5

enum { BC_OUTFLOW = 0, BC_PERIODIC = 1, BC_REFLECT = 2 };
enum { SCHEME_HANCOCK = 0, SCHEME_SSPRK2 = 1, SCHEME_CTU = 2 };
/* what one call of step_with does */
enum { MODE_STAGE = 0, MODE_HANCOCK = 1, MODE_CTU = 2 };
enum { RECON_PLM = 0, RECON_PPM = 1 };
enum { OK = 0, ERR_ARG = -1, ERR_OOM = -2, ERR_NONPHYSICAL = -4 };

typedef struct {
    int ndim;
    int n[3];
    double lo[3], hi[3];
    int bc_lo[3], bc_hi[3];
    double gamma, cfl;
    double grav[3];
    int hse;
    /* hse tables (NULL when hse == 0); centre table index k + 2 for
       k in [-2, nz + 2), face table index f + 2 for the face z_lo + f dz,
       f in [-2, nz + 2]. */
    const double *bg_rho_c, *bg_p_c, *bg_rho_f, *bg_p_f;
    int scheme;     /* SCHEME_HANCOCK or SCHEME_SSPRK2 */
    int recon;      /* RECON_PLM or RECON_PPM */
} orc_params;

/* ------------------------------------------------------------------ */
/* grid bookkeeping                                                    */
/* ------------------------------------------------------------------ */

typedef struct {
    int ndim, nvar;
    int n[3], ng[3], P[3];
    long npad;
    double dx[3];
} grid_t;

static void grid_make(const orc_params *p, grid_t *g)
{
    g->ndim = p->ndim;
    g->nvar = p->ndim + 2;
    g->npad = 1;
    for (int d = 0; d < 3; ++d) {
        g->n[d] = p->n[d];
        g->ng[d] = d < p->ndim ? (p->recon == RECON_PPM ? NG_PPM : NG) : 0;
        g->P[d] = g->n[d] + 2 * g->ng[d];
        g->npad *= g->P[d];
        g->dx[d] = (p->hi[d] - p->lo[d]) / (double)p->n[d];
    }
}

static inline long pidx(const grid_t *g, int i, int j, int k)
{
    return ((long)k * g->P[1] + j) * g->P[0] + i;
}

static int check_params(const orc_params *p)
{
    if (p->ndim < 2 || p->ndim > 3) return ERR_ARG;
    for (int d = 0; d < 3; ++d) {
        if (p->n[d] < 1) return ERR_ARG;
        if (d < p->ndim && p->n[d] < 2) return ERR_ARG;
        if (d >= p->ndim && p->n[d] != 1) return ERR_ARG;
        if (!(p->hi[d] > p->lo[d])) return ERR_ARG;
    }
    if (!(p->gamma > 1.0) || !(p->cfl > 0.0)) return ERR_ARG;
    if (p->scheme != SCHEME_HANCOCK && p->scheme != SCHEME_SSPRK2 && p->scheme != SCHEME_CTU) return ERR_ARG;
    if (p->scheme == SCHEME_CTU && p->recon != RECON_PLM) return ERR_ARG;
    if (p->recon != RECON_PLM && p->recon != RECON_PPM) return ERR_ARG;
    if (p->recon == RECON_PPM) {
        if (p->scheme != SCHEME_SSPRK2 || p->hse) return ERR_ARG;
        for (int d = 0; d < p->ndim; ++d)
            if (p->n[d] < 3) return ERR_ARG;
    }
    if (p->hse) {
        if (p->ndim != 3) return ERR_ARG;
        if (!p->bg_rho_c || !p->bg_p_c || !p->bg_rho_f || !p->bg_p_f) return ERR_ARG;
        if (p->grav[0] != 0.0 || p->grav[1] != 0.0) return ERR_ARG;
    }
    return OK;
}

/* Background at interior z-plane k (may be a ghost plane, k in [-2, nz+2))
   in hse mode; 0 in plain mode. */
static inline double bg_rho_centre(const orc_params *p, int k) { return p->hse ? p->bg_rho_c[k + 2] : 0.0; }
static inline double bg_p_centre(const orc_params *p, int k)   { return p->hse ? p->bg_p_c[k + 2] : 0.0; }
/* face k-1/2 of cell k has face number f = k */
static inline double bg_rho_face(const orc_params *p, int f)   { return p->hse ? p->bg_rho_f[f + 2] : 0.0; }
static inline double bg_p_face(const orc_params *p, int f)     { return p->hse ? p->bg_p_f[f + 2] : 0.0; }

/* ------------------------------------------------------------------ */
/* boundary conditions by index mapping                                */
/* ------------------------------------------------------------------ */

/* Interior source coordinate of padded coordinate c (interior index c-ng)
   along axis d; *flip = 1 when the mapping is a mirror (reflecting wall),
   in which case the normal momentum changes sign. */
static int bc_map(const orc_params *p, const grid_t *g, int d, int c, int *flip)
{
    int n = g->n[d];
    int q = c - g->ng[d];
    *flip = 0;
    if (q >= 0 && q < n) return q;
    if (q < 0) {
        switch (p->bc_lo[d]) {
        case BC_PERIODIC: return q + n;
        case BC_REFLECT: *flip = 1; return -1 - q;
        default: return 0;
        }
    }
    switch (p->bc_hi[d]) {
    case BC_PERIODIC: return q - n;
    case BC_REFLECT: *flip = 1; return 2 * n - 1 - q;
    default: return n - 1;
    }
}

/* Fill the padded conserved array G from the unpadded state U.  Every
   padded cell takes the value of its mapped interior cell; each axis with a
   mirror negates that axis's momentum. */
static void fill_ghosts(const orc_params *p, const grid_t *g, const double *U, double *G)
{
    const long N = (long)g->n[0] * g->n[1] * g->n[2];
    #pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < g->P[2]; ++k)
        for (int j = 0; j < g->P[1]; ++j)
            for (int i = 0; i < g->P[0]; ++i) {
                int fx, fy, fz;
                int si = bc_map(p, g, 0, i, &fx);
                int sj = bc_map(p, g, 1, j, &fy);
                int sk = bc_map(p, g, 2, k, &fz);
                long s = ((long)sk * g->n[1] + sj) * g->n[0] + si;
                long t = pidx(g, i, j, k);
                int flip[3] = {fx, fy, fz};
                for (int q = 0; q < g->nvar; ++q) {
                    double v = U[q * N + s];
                    if (q >= 1 && q <= g->ndim && flip[q - 1]) v = -v;
                    G[q * g->npad + t] = v;
                }
            }
}

/* ------------------------------------------------------------------ */
/* gamma-law EOS                                                       */
/* ------------------------------------------------------------------ */

/* Conserved -> primitive (rho, u_d, p) for one cell.  In hse mode the
   conserved input is the perturbation, rho_bg the background density at the
   cell; the returned density and pressure are perturbations rho', p'. */
static void cons_to_prim(int ndim, double gam, double rho_bg, const double *u, double *w)
{
    double rho_p = u[0];
    double rho = rho_bg + rho_p;
    double m2 = 0.0;
    w[0] = rho_p;
    for (int d = 0; d < ndim; ++d) {
        w[1 + d] = u[1 + d] / rho;
        m2 += u[1 + d] * u[1 + d];
    }
    w[ndim + 1] = (gam - 1.0) * (u[ndim + 1] - 0.5 * m2 / rho);
}

/* Total primitive state -> conserved variables. */
static void prim_to_cons(int ndim, double gam, const double *w, double *u)
{
    double rho = w[0], ke = 0.0;
    u[0] = rho;
    for (int d = 0; d < ndim; ++d) {
        u[1 + d] = rho * w[1 + d];
        ke += w[1 + d] * w[1 + d];
    }
    u[ndim + 1] = w[ndim + 1] / (gam - 1.0) + 0.5 * rho * ke;
}

/* Euler flux along axis d of a total primitive state. */
static void phys_flux(int ndim, double gam, int d, const double *w, double *f)
{
    double rho = w[0], un = w[1 + d], p = w[ndim + 1];
    double ke = 0.0;
    for (int e = 0; e < ndim; ++e) ke += w[1 + e] * w[1 + e];
    double E = p / (gam - 1.0) + 0.5 * rho * ke;
    f[0] = rho * un;
    for (int e = 0; e < ndim; ++e) f[1 + e] = rho * un * w[1 + e];
    f[1 + d] += p;
    f[ndim + 1] = un * (E + p);
}

/* ------------------------------------------------------------------ */
/* MC limiter (van Leer 1977): full-cell slope from left and right   */
/* differences.                                                          */
/* ------------------------------------------------------------------ */

double orc_mc_slope(double dl, double dr)
{
    if (dl * dr <= 0.0) return 0.0;
    double a = fmin(2.0 * fabs(dl), 2.0 * fabs(dr));
    a = fmin(a, 0.5 * fabs(dl + dr));
    return dr > 0.0 ? a : -a;
}

/* ------------------------------------------------------------------ */
/* PPM face values (Colella and Woodward 1984, uniform grid).  am, a, ap:  */
/* the values of cells i-1, i, i+1; sm, s, sp: their MC-limited slopes.    */
/* Returns the limited parabola's values at the low and high faces of i.   */
/* ------------------------------------------------------------------ */

void orc_ppm_faces(double am, double a, double ap, double sm, double s, double sp,
                   double *lo, double *hi)
{
    /* interface values (their eq. 1.9 with the limited slopes of eq. 1.8) */
    double aL = 0.5 * (am + a) - (s - sm) / 6.0;
    double aR = 0.5 * (a + ap) - (sp - s) / 6.0;
    /* monotone parabola (their eq. 1.10) */
    if ((aR - a) * (a - aL) <= 0.0) {
        aL = a;
        aR = a;
    } else {
        double da = aR - aL;
        double a6 = 6.0 * (a - 0.5 * (aL + aR));
        if (da * a6 > da * da) aL = 3.0 * a - 2.0 * aR;
        else if (-(da * da) > da * a6) aR = 3.0 * a - 2.0 * aL;
    }
    *lo = aL;
    *hi = aR;
}

static void ppm_faces(double am, double a, double ap, double sm, double s, double sp,
                      double *lo, double *hi)
{
    orc_ppm_faces(am, a, ap, sm, s, sp, lo, hi);
}

/* ------------------------------------------------------------------ */
/* HLLC flux (Toro, Riemann Solvers and Numerical Methods for Fluid  */
/* Dynamics, 3rd ed., sec. 10.4-10.6) with Davis wave-speed estimates,  */
/* states in total primitive variables, branch tie S* = 0 to the left.  */
/* ------------------------------------------------------------------ */

void orc_hllc(int ndim, double gam, int d, const double *wl, const double *wr, double *f)
{
    const int nv = ndim + 2;
    double rl = wl[0], ul = wl[1 + d], pl = wl[ndim + 1];
    double rr = wr[0], ur = wr[1 + d], pr = wr[ndim + 1];
    double cl = sqrt(gam * pl / rl);
    double cr = sqrt(gam * pr / rr);
    double sl = fmin(ul - cl, ur - cr);
    double sr = fmax(ul + cl, ur + cr);
    double fl[MAXV], fr[MAXV], ucl[MAXV], ucr[MAXV];
    phys_flux(ndim, gam, d, wl, fl);
    phys_flux(ndim, gam, d, wr, fr);
    if (0.0 <= sl) { memcpy(f, fl, nv * sizeof(double)); return; }
    if (sr <= 0.0) { memcpy(f, fr, nv * sizeof(double)); return; }
    double sstar = (pr - pl + rl * ul * (sl - ul) - rr * ur * (sr - ur))
                 / (rl * (sl - ul) - rr * (sr - ur));
    prim_to_cons(ndim, gam, wl, ucl);
    prim_to_cons(ndim, gam, wr, ucr);
    const double *w = sstar >= 0.0 ? wl : wr;
    const double *uk = sstar >= 0.0 ? ucl : ucr;
    const double *fk = sstar >= 0.0 ? fl : fr;
    double sk = sstar >= 0.0 ? sl : sr;
    double rk = w[0], uk_n = w[1 + d], pk = w[ndim + 1];
    /* star state U*_K (Toro eq. 10.39) */
    double fac = rk * (sk - uk_n) / (sk - sstar);
    double ustar[MAXV];
    ustar[0] = fac;
    for (int e = 0; e < ndim; ++e) ustar[1 + e] = fac * w[1 + e];
    ustar[1 + d] = fac * sstar;
    ustar[ndim + 1] = fac * (uk[ndim + 1] / rk
                             + (sstar - uk_n) * (sstar + pk / (rk * (sk - uk_n))));
    /* F*_K = F_K + S_K (U*_K - U_K) (Toro eq. 10.38) */
    for (int q = 0; q < nv; ++q) f[q] = fk[q] + sk * (ustar[q] - uk[q]);
}

/* ------------------------------------------------------------------ */
/* CFL time step                                                       */
/* ------------------------------------------------------------------ */

/* max over cells of sum_d (|u_d| + c) / dx_d for an unpadded state */
double orc_max_signal(const orc_params *p, const double *U)
{
    grid_t g;
    grid_make(p, &g);
    const long N = (long)g.n[0] * g.n[1] * g.n[2];
    double smax = 0.0;
    #pragma omp parallel for collapse(2) reduction(max : smax) schedule(static)
    for (int k = 0; k < g.n[2]; ++k)
        for (int j = 0; j < g.n[1]; ++j) {
            double rho_bg = bg_rho_centre(p, k), p_bg = bg_p_centre(p, k);
            for (int i = 0; i < g.n[0]; ++i) {
                long c = ((long)k * g.n[1] + j) * g.n[0] + i;
                double u[MAXV], w[MAXV];
                for (int q = 0; q < g.nvar; ++q) u[q] = U[q * N + c];
                cons_to_prim(g.ndim, p->gamma, rho_bg, u, w);
                double rho = rho_bg + w[0];
                double pr = p_bg + w[g.ndim + 1];
                double cs = sqrt(p->gamma * pr / rho);
                double s = 0.0;
                for (int d = 0; d < g.ndim; ++d) s += (fabs(w[1 + d]) + cs) / g.dx[d];
                if (s > smax) smax = s;
            }
        }
    return smax;
}

double orc_cfl_dt(const orc_params *p, const double *U)
{
    return p->cfl / orc_max_signal(p, U);
}

/* ------------------------------------------------------------------ */
/* one step                                                             */
/* ------------------------------------------------------------------ */

typedef struct {
    grid_t g;
    double *G;      /* padded conserved (perturbation in hse mode)   nvar    */
    double *W;      /* padded primitives (rho', u, p')               nvar    */
    double *dW;     /* MC slopes, [d][q]                             ndim*nvar */
    double *Wf;     /* face states, [d][side][q]; side 0 = low face  2*ndim*nvar */
    double *F;      /* fluxes through the high face of each cell, [d][q] */
    double *F1;     /* corner transport upwind: first-pass fluxes, [d][q] */
    unsigned char *fb;  /* 1 where a cell's face states took the positivity fallback */
} work_t;

/* Test instrumentation (no effect on any result): interior cells whose face
   states took the positivity fallback (slopes zeroed), and cell-axis pairs
   of the corner transport upwind step kept uncorrected, summed over every
   step since the last orc_fallback_counts(.., 1). */
static long long fallback_cells = 0, ctu_uncorrected_pairs = 0;

static void work_free(work_t *w)
{
    free(w->G); free(w->W); free(w->dW); free(w->Wf); free(w->F); free(w->F1); free(w->fb);
    memset(w, 0, sizeof(*w));
}

static int work_alloc(const orc_params *p, work_t *w)
{
    memset(w, 0, sizeof(*w));
    grid_make(p, &w->g);
    size_t a = (size_t)w->g.npad * sizeof(double);
    int nv = w->g.nvar, nd = w->g.ndim;
    w->G = (double *)calloc((size_t)nv, a);
    w->W = (double *)calloc((size_t)nv, a);
    w->dW = (double *)calloc((size_t)nd * nv, a);
    w->Wf = (double *)calloc((size_t)2 * nd * nv, a);
    w->F = (double *)calloc((size_t)nd * nv, a);
    w->fb = (unsigned char *)calloc((size_t)w->g.npad, 1);
    if (!w->fb) { work_free(w); return ERR_OOM; }
    if (p->scheme == SCHEME_CTU) {
        w->F1 = (double *)calloc((size_t)nd * nv, a);
        if (!w->F1) { work_free(w); return ERR_OOM; }
    }
    if (!w->G || !w->W || !w->dW || !w->Wf || !w->F) { work_free(w); return ERR_OOM; }
    return OK;
}

/* padded z-plane kk -> interior plane index k (may be outside [0, nz)) */
static inline int zplane(const grid_t *g, int kk) { return kk - g->ng[2]; }

/* HLLC flux through the high face of each cell along every axis d, from
   the face states Wf, into F.  ext = 0: the faces of the interior (cells
   ng-1 .. ng+n-1 along d, interior across); ext = 1: also one ring of cells
   beyond the interior across d (the first pass of the corner transport
   upwind method). */
static void flux_pass(const orc_params *p, work_t *wk, const double *Wf, double *F, int ext)
{
    const grid_t *g = &wk->g;
    const int nd = g->ndim, nv = g->nvar;
    const long np = g->npad;
    const double gam = p->gamma;
    const int st[3] = {1, g->P[0], g->P[0] * g->P[1]};
    for (int d = 0; d < nd; ++d) {
        int flo[3], fhi[3];
        for (int e = 0; e < 3; ++e) {
            int x = (ext && e != d && g->ng[e] > 0) ? 1 : 0;
            flo[e] = g->ng[e] - x;
            fhi[e] = g->ng[e] + g->n[e] + x;
        }
        flo[d] -= 1;
        #pragma omp parallel for collapse(2) schedule(static)
        for (int kk = flo[2]; kk < fhi[2]; ++kk)
            for (int j = flo[1]; j < fhi[1]; ++j) {
                int k = zplane(g, kk);
                for (int i = flo[0]; i < fhi[0]; ++i) {
                    long c = pidx(g, i, j, kk);
                    long cn = c + st[d];
                    double wl[MAXV], wr[MAXV], f[MAXV];
                    /* background at this face: the z face k+1/2, or the
                       plane's centre value for x and y faces */
                    double rb, pb;
                    if (d == 2) { rb = bg_rho_face(p, k + 1); pb = bg_p_face(p, k + 1); }
                    else        { rb = bg_rho_centre(p, k);   pb = bg_p_centre(p, k); }
                    for (int q = 0; q < nv; ++q) {
                        wl[q] = Wf[((d * 2 + 1) * nv + q) * np + c];
                        wr[q] = Wf[((d * 2 + 0) * nv + q) * np + cn];
                    }
                    /* reflecting wall: the far side of the wall face is the
                       mirror image of the interior cell's predicted face
                       state (normal velocity negated), so no mass crosses it */
                    int cd = d == 0 ? i : (d == 1 ? j : kk);
                    if (cd == g->ng[d] - 1 && p->bc_lo[d] == BC_REFLECT) {
                        for (int q = 0; q < nv; ++q) wl[q] = wr[q];
                        wl[1 + d] = -wr[1 + d];
                    }
                    if (cd == g->ng[d] + g->n[d] - 1 && p->bc_hi[d] == BC_REFLECT) {
                        for (int q = 0; q < nv; ++q) wr[q] = wl[q];
                        wr[1 + d] = -wl[1 + d];
                    }
                    wl[0] += rb; wr[0] += rb;
                    wl[nd + 1] += pb; wr[nd + 1] += pb;
                    orc_hllc(nd, gam, d, wl, wr, f);
                    f[1 + d] -= pb;   /* momentum flux carries p' */
                    for (int q = 0; q < nv; ++q) F[(d * nv + q) * np + c] = f[q];
                }
            }
    }
}

/* Corner transport upwind: correct the face states of every cell that
   borders an interior face along d (cells ng-1 .. ng+n along d, interior
   across) by the transverse differences of the first-pass fluxes of that
   cell, in conserved variables; a cell whose corrected pair along d has a
   non-positive density or pressure keeps its uncorrected pair. */
static void ctu_correct(const orc_params *p, work_t *wk, double dt)
{
    const grid_t *g = &wk->g;
    const int nd = g->ndim, nv = g->nvar;
    const long np = g->npad;
    const int st[3] = {1, g->P[0], g->P[0] * g->P[1]};
    for (int d = 0; d < nd; ++d) {
        int clo[3], chi[3];
        for (int e = 0; e < 3; ++e) {
            clo[e] = g->ng[e];
            chi[e] = g->ng[e] + g->n[e];
        }
        clo[d] -= 1;
        chi[d] += 1;
        long long kept = 0;
        #pragma omp parallel for collapse(2) schedule(static) reduction(+ : kept)
        for (int kk = clo[2]; kk < chi[2]; ++kk)
            for (int j = clo[1]; j < chi[1]; ++j)
                for (int i = clo[0]; i < chi[0]; ++i) {
                    long c = pidx(g, i, j, kk);
                    double wc[2][MAXV];
                    int bad = 0;
                    /* background at the two faces: the plane's centre value for x
                       and y faces, the face values for z faces (hse mode) */
                    const int k = zplane(g, kk);
                    for (int s = 0; s < 2; ++s) {
                        double rb = bg_rho_centre(p, k), pb = bg_p_centre(p, k);
                        if (d == 2) { rb = bg_rho_face(p, k + s); pb = bg_p_face(p, k + s); }
                        double w[MAXV], u[MAXV];
                        for (int q = 0; q < nv; ++q) w[q] = wk->Wf[((d * 2 + s) * nv + q) * np + c];
                        w[0] += rb;
                        w[nd + 1] += pb;
                        prim_to_cons(nd, p->gamma, w, u);
                        for (int e = 0; e < nd; ++e) {
                            if (e == d) continue;
                            for (int q = 0; q < nv; ++q) {
                                const double *Fq = wk->F1 + (e * nv + q) * np;
                                u[q] -= dt / (2.0 * g->dx[e]) * (Fq[c] - Fq[c - st[e]]);
                            }
                            /* hse: the z fluxes carry p'; the correction of a
                               total state needs the background's pressure too */
                            if (p->hse && e == 2)
                                u[3] -= dt / (2.0 * g->dx[2]) * (bg_p_face(p, k + 1) - bg_p_face(p, k));
                        }
                        cons_to_prim(nd, p->gamma, 0.0, u, wc[s]);
                        if (!(wc[s][0] > 0.0) || !(wc[s][nd + 1] > 0.0)) bad = 1;
                        wc[s][0] -= rb;
                        wc[s][nd + 1] -= pb;
                    }
                    if (bad) { ++kept; continue; }
                    for (int s = 0; s < 2; ++s)
                        for (int q = 0; q < nv; ++q) wk->Wf[((d * 2 + s) * nv + q) * np + c] = wc[s][q];
                }
        ctu_uncorrected_pairs += kept;
    }
}

/* One update U <- U + dt * (flux divergence + sources).  mode MODE_HANCOCK:
   the MUSCL-Hancock step; MODE_STAGE: one forward-Euler stage U + dt L(U)
   of the method of lines (face states W -/+ dW/2, gravity on the momentum
   from the stage density); MODE_CTU: the corner transport upwind step. */
static void predict_faces(const orc_params *p, work_t *wk, const double *U, double dt, int mode)
{
    const int predictor = mode != MODE_STAGE;
    const grid_t *g = &wk->g;
    const int nd = g->ndim, nv = g->nvar;
    const long np = g->npad;
    const double gam = p->gamma;
    const int st[3] = {1, g->P[0], g->P[0] * g->P[1]};   /* padded strides */

    /* 1. ghost cells */
    fill_ghosts(p, g, U, wk->G);

    /* 2. primitives on every padded cell */
    #pragma omp parallel for collapse(2) schedule(static)
    for (int kk = 0; kk < g->P[2]; ++kk)
        for (int j = 0; j < g->P[1]; ++j) {
            double rho_bg = bg_rho_centre(p, zplane(g, kk));
            for (int i = 0; i < g->P[0]; ++i) {
                long c = pidx(g, i, j, kk);
                double u[MAXV], w[MAXV];
                for (int q = 0; q < nv; ++q) u[q] = wk->G[q * np + c];
                cons_to_prim(nd, gam, rho_bg, u, w);
                for (int q = 0; q < nv; ++q) wk->W[q * np + c] = w[q];
            }
        }

    /* cells that need slopes: every padded cell with both neighbours along
       each active axis; cells that need face states: one ring beyond the
       interior (the same cells for PLM's two ghosts) */
    int lo[3], hi[3], flo_c[3], fhi_c[3];
    for (int d = 0; d < 3; ++d) {
        lo[d] = g->ng[d] > 0 ? 1 : 0;
        hi[d] = g->ng[d] > 0 ? g->P[d] - 1 : g->P[d];   /* exclusive */
        flo_c[d] = g->ng[d] > 0 ? g->ng[d] - 1 : 0;
        fhi_c[d] = g->ng[d] > 0 ? g->ng[d] + g->n[d] + 1 : g->P[d];
    }

    /* 3. MC slopes of each primitive along each axis */
    #pragma omp parallel for collapse(2) schedule(static)
    for (int kk = lo[2]; kk < hi[2]; ++kk)
        for (int j = lo[1]; j < hi[1]; ++j)
            for (int i = lo[0]; i < hi[0]; ++i) {
                long c = pidx(g, i, j, kk);
                for (int d = 0; d < nd; ++d)
                    for (int q = 0; q < nv; ++q) {
                        const double *Wq = wk->W + q * np;
                        double dl = Wq[c] - Wq[c - st[d]];
                        double dr = Wq[c + st[d]] - Wq[c];
                        wk->dW[(d * nv + q) * np + c] = orc_mc_slope(dl, dr);
                    }
            }

    /* 4. MUSCL-Hancock half step in primitive variables, all axes
       at once, then face states W +- dW/2 (or PPM's) with the per-cell
       fallback */
    const double hdt = 0.5 * dt;
    long long nfb = 0;
    #pragma omp parallel for collapse(2) schedule(static) reduction(+ : nfb)
    for (int kk = flo_c[2]; kk < fhi_c[2]; ++kk)
        for (int j = flo_c[1]; j < fhi_c[1]; ++j) {
            int k = zplane(g, kk);
            double rho_bg = bg_rho_centre(p, k), p_bg = bg_p_centre(p, k);
            /* background slopes and discrete imbalance across the cell (z) */
            double drho_bg = bg_rho_face(p, k + 1) - bg_rho_face(p, k);
            double dp_bg = bg_p_face(p, k + 1) - bg_p_face(p, k);
            double B = p->hse ? dp_bg / g->dx[2] - rho_bg * p->grav[2] : 0.0;
            for (int i = flo_c[0]; i < fhi_c[0]; ++i) {
                long c = pidx(g, i, j, kk);
                double w[MAXV], dw[3][MAXV], wh[MAXV];
                for (int q = 0; q < nv; ++q) w[q] = wk->W[q * np + c];
                for (int d = 0; d < nd; ++d)
                    for (int q = 0; q < nv; ++q) dw[d][q] = wk->dW[(d * nv + q) * np + c];
                double rho = rho_bg + w[0];
                double pr = p_bg + w[nd + 1];
                /* time derivative of W from A_d(W) dW_d / dx_d, summed over d */
                double dwdt[MAXV] = {0};
                for (int d = 0; d < nd; ++d) {
                    double un = w[1 + d];
                    dwdt[0] -= (un * dw[d][0] + rho * dw[d][1 + d]) / g->dx[d];
                    for (int e = 0; e < nd; ++e) dwdt[1 + e] -= un * dw[d][1 + e] / g->dx[d];
                    dwdt[1 + d] -= dw[d][nd + 1] / rho / g->dx[d];
                    dwdt[nd + 1] -= (un * dw[d][nd + 1] + gam * pr * dw[d][1 + d]) / g->dx[d];
                }
                if (p->hse) {  /* background advection and pressure terms */
                    double wz = w[3];
                    dwdt[0] -= wz * drho_bg / g->dx[2];
                    dwdt[4] -= wz * dp_bg / g->dx[2];
                    dwdt[3] -= B / rho;
                }
                /* gravity: du/dt = g (rho' / rho); rho'/rho = 1 in plain mode */
                for (int d = 0; d < nd; ++d) dwdt[1 + d] += p->grav[d] * (w[0] / rho);
                if (predictor)
                    for (int q = 0; q < nv; ++q) wh[q] = w[q] + hdt * dwdt[q];
                else
                    for (int q = 0; q < nv; ++q) wh[q] = w[q];
                /* corner transport upwind: per axis the one-dimensional
                   predictor, only that axis's A_d term plus gravity */
                double wd[3][MAXV];
                if (mode == MODE_CTU)
                    for (int d = 0; d < nd; ++d) {
                        double r[MAXV] = {0};
                        double un = w[1 + d];
                        r[0] = -(un * dw[d][0] + rho * dw[d][1 + d]) / g->dx[d];
                        for (int e = 0; e < nd; ++e) r[1 + e] = -un * dw[d][1 + e] / g->dx[d];
                        r[1 + d] -= dw[d][nd + 1] / rho / g->dx[d];
                        r[nd + 1] = -(un * dw[d][nd + 1] + gam * pr * dw[d][1 + d]) / g->dx[d];
                        if (p->hse && d == 2) {   /* advection of the background along z */
                            r[0] -= w[3] * drho_bg / g->dx[2];
                            r[4] -= w[3] * dp_bg / g->dx[2];
                        }
                        /* gravity on the velocities in every axis's predictor: g,
                           except in the z predictor of hse mode, which takes the
                           background's pressure gradient from its imbalance
                           instead (g rho'/rho - B/rho) */
                        const double gf = (p->hse && d == 2) ? w[0] / rho : 1.0;
                        for (int e = 0; e < nd; ++e) r[1 + e] += p->grav[e] * gf;
                        if (p->hse && d == 2) r[3] -= B / rho;
                        for (int q = 0; q < nv; ++q) wd[d][q] = w[q] + hdt * r[q];
                    }

                double wf[3][2][MAXV];
                int bad = 0;
                if (p->recon == RECON_PPM) {
                    for (int d = 0; d < nd; ++d)
                        for (int q = 0; q < nv; ++q) {
                            const double *Wq = wk->W + q * np;
                            const double *Dq = wk->dW + (d * nv + q) * np;
                            ppm_faces(Wq[c - st[d]], Wq[c], Wq[c + st[d]], Dq[c - st[d]], Dq[c],
                                      Dq[c + st[d]], &wf[d][0][q], &wf[d][1][q]);
                        }
                }
                for (int d = 0; d < nd; ++d)
                    for (int s = 0; s < 2; ++s) {
                        double sgn = s == 0 ? -0.5 : 0.5;
                        if (mode == MODE_CTU)
                            for (int q = 0; q < nv; ++q) wf[d][s][q] = wd[d][q] + sgn * dw[d][q];
                        else if (p->recon == RECON_PLM)
                            for (int q = 0; q < nv; ++q) wf[d][s][q] = wh[q] + sgn * dw[d][q];
                        /* totals at this face for the positivity test */
                        double rb = rho_bg, pb = p_bg;
                        if (p->hse && d == 2) {
                            rb = bg_rho_face(p, k + s);
                            pb = bg_p_face(p, k + s);
                        }
                        if (!(rb + wf[d][s][0] > 0.0) || !(pb + wf[d][s][nd + 1] > 0.0)) bad = 1;
                    }
                if (bad) {
                    /* positivity fallback: zero every slope of this cell */
                    double w0[MAXV];
                    for (int q = 0; q < nv; ++q) w0[q] = w[q];
                    if (predictor) {
                        for (int d = 0; d < nd; ++d) w0[1 + d] += hdt * p->grav[d] * (w[0] / rho);
                        if (p->hse) w0[3] -= hdt * B / rho;
                    }
                    for (int d = 0; d < nd; ++d)
                        for (int s = 0; s < 2; ++s)
                            for (int q = 0; q < nv; ++q) wf[d][s][q] = w0[q];
                    if (mode == MODE_CTU && p->hse)   /* x and y states: plain gravity (as their predictor) */
                        for (int d = 0; d < nd && d < 2; ++d)
                            for (int s = 0; s < 2; ++s)
                                for (int e = 0; e < nd; ++e) wf[d][s][1 + e] = w[1 + e] + hdt * p->grav[e];
                }
                for (int d = 0; d < nd; ++d)
                    for (int s = 0; s < 2; ++s)
                        for (int q = 0; q < nv; ++q)
                            wk->Wf[((d * 2 + s) * nv + q) * np + c] = wf[d][s][q];
                wk->fb[c] = (unsigned char)bad;
                if (bad && i >= g->ng[0] && i < g->ng[0] + g->n[0] && j >= g->ng[1] &&
                    j < g->ng[1] + g->n[1] && kk >= g->ng[2] && kk < g->ng[2] + g->n[2])
                    ++nfb;
            }
        }
    fallback_cells += nfb;
}

static int step_with(const orc_params *p, work_t *wk, double *U, double dt, int mode)
{
    const int predictor = mode != MODE_STAGE;
    const grid_t *g = &wk->g;
    const int nd = g->ndim, nv = g->nvar;
    const long np = g->npad;
    const long N = (long)g->n[0] * g->n[1] * g->n[2];
    const double gam = p->gamma;
    const int st[3] = {1, g->P[0], g->P[0] * g->P[1]};

    /* 1.-4. ghosts, primitives, slopes, predicted face states */
    predict_faces(p, wk, U, dt, mode);

    /* 5. HLLC flux through the high face of each cell along d, for every
       face of the interior; the corner transport upwind step first takes
       fluxes from the one-dimensional states (one ring wider) and corrects
       the states with their transverse differences */
    if (mode == MODE_CTU) {
        flux_pass(p, wk, wk->Wf, wk->F1, 1);
        ctu_correct(p, wk, dt);
    }
    flux_pass(p, wk, wk->Wf, wk->F, 0);

    /* 6. conservative update, density first, then momentum with
       the time-centred density in the gravity source (MUSCL-Hancock) or the
       stage density (method of lines), then energy with the mass fluxes
       through the two faces */
    int bad_total = 0;
    #pragma omp parallel for collapse(2) schedule(static) reduction(| : bad_total)
    for (int k = 0; k < g->n[2]; ++k)
        for (int j = 0; j < g->n[1]; ++j) {
            int kk = k + g->ng[2];
            double rho_bg = bg_rho_centre(p, k);
            double B = 0.0;
            if (p->hse)
                B = (bg_p_face(p, k + 1) - bg_p_face(p, k)) / g->dx[2] - rho_bg * p->grav[2];
            for (int i = 0; i < g->n[0]; ++i) {
                long c = pidx(g, i + g->ng[0], j + g->ng[1], kk);
                long o = ((long)k * g->n[1] + j) * g->n[0] + i;
                double du[MAXV] = {0};
                double mass_src = 0.0;   /* sum_d g_d (F_rho,lo + F_rho,hi) / 2 */
                for (int d = 0; d < nd; ++d) {
                    for (int q = 0; q < nv; ++q) {
                        const double *Fq = wk->F + (d * nv + q) * np;
                        du[q] -= (Fq[c] - Fq[c - st[d]]) / g->dx[d];
                    }
                    const double *Fr = wk->F + (d * nv + 0) * np;
                    mass_src += p->grav[d] * 0.5 * (Fr[c - st[d]] + Fr[c]);
                }
                double rho_old = U[0 * N + o];
                double rho_new = rho_old + dt * du[0];
                U[0 * N + o] = rho_new;
                for (int d = 0; d < nd; ++d) {
                    double src = predictor ? p->grav[d] * 0.5 * (rho_old + rho_new)
                                           : p->grav[d] * rho_old;
                    if (p->hse && d == 2) src -= B;
                    U[(1 + d) * N + o] += dt * (du[1 + d] + src);
                }
                U[(nd + 1) * N + o] += dt * (du[nd + 1] + mass_src);
                /* physical admissibility of the new state */
                double u[MAXV], w[MAXV];
                for (int q = 0; q < nv; ++q) u[q] = U[q * N + o];
                cons_to_prim(nd, gam, rho_bg, u, w);
                double rt = rho_bg + w[0], pt = bg_p_centre(p, k) + w[nd + 1];
                if (!(rt > 0.0) || !(pt > 0.0) || !isfinite(rt) || !isfinite(pt)) bad_total |= 1;
            }
        }
    return bad_total ? ERR_NONPHYSICAL : OK;
}

/* ------------------------------------------------------------------ */
/* public entry points                                                  */
/* ------------------------------------------------------------------ */

void orc_set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* One full step of the problem's integrator with the given dt. */
static int full_step(const orc_params *p, work_t *wk, double *U, double *U0, double dt)
{
    if (p->scheme == SCHEME_HANCOCK) return step_with(p, wk, U, dt, MODE_HANCOCK);
    if (p->scheme == SCHEME_CTU) return step_with(p, wk, U, dt, MODE_CTU);
    /* SSP-RK2: U0 keeps U^n; U becomes U1, then U1 + dt L(U1), then the
       average with U^n */
    const long n = (long)wk->g.nvar * wk->g.n[0] * wk->g.n[1] * wk->g.n[2];
    memcpy(U0, U, sizeof(double) * n);
    int rc1 = step_with(p, wk, U, dt, MODE_STAGE);   /* checks U1 */
    step_with(p, wk, U, dt, MODE_STAGE);             /* U1 + dt L(U1): only its average is a state */
    for (long i = 0; i < n; ++i) U[i] = 0.5 * (U0[i] + U[i]);
    /* admissibility of U^{n+1} */
    const grid_t *g = &wk->g;
    const long N = (long)g->n[0] * g->n[1] * g->n[2];
    int bad = 0;
    for (int k = 0; k < g->n[2]; ++k)
        for (int j = 0; j < g->n[1]; ++j)
            for (int i = 0; i < g->n[0]; ++i) {
                long c = ((long)k * g->n[1] + j) * g->n[0] + i;
                double u[MAXV], w[MAXV];
                for (int q = 0; q < g->nvar; ++q) u[q] = U[q * N + c];
                cons_to_prim(g->ndim, p->gamma, bg_rho_centre(p, k), u, w);
                double rt = bg_rho_centre(p, k) + w[0], pt = bg_p_centre(p, k) + w[g->ndim + 1];
                if (!(rt > 0.0) || !(pt > 0.0) || !isfinite(rt) || !isfinite(pt)) bad = 1;
            }
    return rc1 ? rc1 : bad ? ERR_NONPHYSICAL : OK;
}

int orc_step(const orc_params *p, double *U, double dt)
{
    int rc = check_params(p);
    if (rc) return rc;
    work_t wk;
    if (work_alloc(p, &wk)) return ERR_OOM;
    double *U0 = (double *)malloc(sizeof(double) * wk.g.nvar * wk.g.n[0] * wk.g.n[1] * wk.g.n[2]);
    if (!U0) { work_free(&wk); return ERR_OOM; }
    rc = full_step(p, &wk, U, U0, dt);
    free(U0);
    work_free(&wk);
    return rc;
}

/* Advance U from time t0 until t_end or max_steps steps: each step
   takes dt = cfl / max signal speed of the current state, clamped to land
   exactly on t_end.  Writes the final time, the step count and the last dt
   taken.  dts (nullable, max_steps long) receives every dt taken. */
int orc_run(const orc_params *p, double *U, double t0, double t_end, long max_steps,
            double *t_out, long *steps_out, double *dt_last_out, double *dts)
{
    int rc = check_params(p);
    if (rc) return rc;
    work_t wk;
    if (work_alloc(p, &wk)) return ERR_OOM;
    double *U0 = (double *)malloc(sizeof(double) * wk.g.nvar * wk.g.n[0] * wk.g.n[1] * wk.g.n[2]);
    if (!U0) { work_free(&wk); return ERR_OOM; }
    double t = t0, dt_last = 0.0;
    long s = 0;
    while (s < max_steps && t < t_end) {
        double dt = orc_cfl_dt(p, U);
        double tn;
        if (dt >= t_end - t) { dt = t_end - t; tn = t_end; }
        else tn = t + dt;
        rc = full_step(p, &wk, U, U0, dt);
        if (dts) dts[s] = dt;
        t = tn;
        dt_last = dt;
        ++s;
        if (rc) break;
    }
    free(U0);
    work_free(&wk);
    if (t_out) *t_out = t;
    if (steps_out) *steps_out = s;
    if (dt_last_out) *dt_last_out = dt_last;
    return rc;
}

/* Primitive (total) -> conserved for a whole state; in hse mode the
   background of each plane is subtracted to give the stored perturbation. */
int orc_prim_to_state(const orc_params *p, const double *W, double *U)
{
    int rc = check_params(p);
    if (rc) return rc;
    grid_t g;
    grid_make(p, &g);
    const long N = (long)g.n[0] * g.n[1] * g.n[2];
    for (int k = 0; k < g.n[2]; ++k)
        for (long c = (long)k * g.n[0] * g.n[1]; c < (long)(k + 1) * g.n[0] * g.n[1]; ++c) {
            double w[MAXV], u[MAXV];
            for (int q = 0; q < g.nvar; ++q) w[q] = W[q * N + c];
            prim_to_cons(g.ndim, p->gamma, w, u);
            u[0] -= bg_rho_centre(p, k);
            u[g.nvar - 1] -= bg_p_centre(p, k) / (p->gamma - 1.0);
            for (int q = 0; q < g.nvar; ++q) U[q * N + c] = u[q];
        }
    return OK;
}

/* Stored state -> total conserved variables (adds the background back). */
int orc_state_to_total(const orc_params *p, const double *U, double *T)
{
    int rc = check_params(p);
    if (rc) return rc;
    grid_t g;
    grid_make(p, &g);
    const long N = (long)g.n[0] * g.n[1] * g.n[2];
    const long plane = (long)g.n[0] * g.n[1];
    for (int k = 0; k < g.n[2]; ++k)
        for (long c = k * plane; c < (k + 1) * plane; ++c) {
            for (int q = 0; q < g.nvar; ++q) T[q * N + c] = U[q * N + c];
            T[c] += bg_rho_centre(p, k);
            T[(g.nvar - 1) * N + c] += bg_p_centre(p, k) / (p->gamma - 1.0);
        }
    return OK;
}

/* Stored state -> total primitive variables (rho, u_d, p). */
int orc_state_to_prim(const orc_params *p, const double *U, double *W)
{
    int rc = check_params(p);
    if (rc) return rc;
    grid_t g;
    grid_make(p, &g);
    const long N = (long)g.n[0] * g.n[1] * g.n[2];
    const long plane = (long)g.n[0] * g.n[1];
    for (int k = 0; k < g.n[2]; ++k)
        for (long c = k * plane; c < (k + 1) * plane; ++c) {
            double u[MAXV], w[MAXV];
            for (int q = 0; q < g.nvar; ++q) u[q] = U[q * N + c];
            cons_to_prim(g.ndim, p->gamma, bg_rho_centre(p, k), u, w);
            w[0] += bg_rho_centre(p, k);
            w[g.nvar - 1] += bg_p_centre(p, k);
            for (int q = 0; q < g.nvar; ++q) W[q * N + c] = w[q];
        }
    return OK;
}

/* conserved totals sum_cells q dV of the TOTAL state, in plain
   sequential order (cell volume applied once at the end). */
int orc_totals(const orc_params *p, const double *U, double *out)
{
    int rc = check_params(p);
    if (rc) return rc;
    grid_t g;
    grid_make(p, &g);
    const long N = (long)g.n[0] * g.n[1] * g.n[2];
    const long plane = (long)g.n[0] * g.n[1];
    double dV = 1.0;
    for (int d = 0; d < g.ndim; ++d) dV *= g.dx[d];
    for (int q = 0; q < g.nvar; ++q) {
        double s = 0.0;
        for (int k = 0; k < g.n[2]; ++k) {
            double bg = 0.0;
            if (q == 0) bg = bg_rho_centre(p, k);
            if (q == g.nvar - 1) bg = bg_p_centre(p, k) / (p->gamma - 1.0);
            for (long c = k * plane; c < (k + 1) * plane; ++c) s += U[q * N + c] + bg;
        }
        out[q] = s * dV;
    }
    return OK;
}

/* Single-face helpers for unit tests. */
void orc_phys_flux(int ndim, double gam, int d, const double *w, double *f)
{
    phys_flux(ndim, gam, d, w, f);
}

void orc_prim_to_cons1(int ndim, double gam, const double *w, double *u)
{
    prim_to_cons(ndim, gam, w, u);
}

/* ------------------------------------------------------------------ */
/* test instrumentation                                                 */
/* ------------------------------------------------------------------ */

/* out[0]: interior cells whose face states took the positivity fallback,
   out[1]: corner transport upwind cell-axis pairs kept uncorrected, both
   summed over every step since the last reset; reset != 0 zeroes them
   after reading. */
void orc_fallback_counts(long long *out, int reset)
{
    out[0] = fallback_cells;
    out[1] = ctu_uncorrected_pairs;
    if (reset) fallback_cells = ctu_uncorrected_pairs = 0;
}

/* The face states the problem's integrator predicts from U with time step
   dt (steps 1-4 of a step; for the corner transport upwind method the
   one-dimensional predictor's states before the transverse correction; for
   the method of lines the first stage's W -/+ dW/2), for every interior
   cell: Wf[((d * 2 + s) * nvar + q) * N + cell], s = 0 the low face, in
   the stored form (rho', u, p' in hse mode); mask[cell] = 1 where the cell
   took the positivity fallback. */
int orc_face_states(const orc_params *p, const double *U, double dt, double *Wf, unsigned char *mask)
{
    int rc = check_params(p);
    if (rc) return rc;
    work_t wk;
    if (work_alloc(p, &wk)) return ERR_OOM;
    const int mode = p->scheme == SCHEME_CTU ? MODE_CTU : (p->scheme == SCHEME_SSPRK2 ? MODE_STAGE : MODE_HANCOCK);
    predict_faces(p, &wk, U, dt, mode);
    const grid_t *g = &wk.g;
    const int nd = g->ndim, nv = g->nvar;
    const long np = g->npad, N = (long)g->n[0] * g->n[1] * g->n[2];
    for (int k = 0; k < g->n[2]; ++k)
        for (int j = 0; j < g->n[1]; ++j)
            for (int i = 0; i < g->n[0]; ++i) {
                long c = pidx(g, i + g->ng[0], j + g->ng[1], k + g->ng[2]);
                long o = ((long)k * g->n[1] + j) * g->n[0] + i;
                for (int d = 0; d < nd; ++d)
                    for (int s = 0; s < 2; ++s)
                        for (int q = 0; q < nv; ++q)
                            Wf[((long)(d * 2 + s) * nv + q) * N + o] = wk.Wf[((d * 2 + s) * nv + q) * np + c];
                mask[o] = wk.fb[c];
            }
    work_free(&wk);
    return OK;
}
