/*
 * exact_riemann.c -- TEST INFRASTRUCTURE ONLY.
 *
 * Exact solution of the Riemann problem for the 1D Euler equations of a
 * gamma-law gas, following the mathematics of Toro, "Riemann Solvers and
 * Numerical Methods for Fluid Dynamics", 3rd ed., chapter 4:
 *   - the star pressure p* is the root of f_L(p) + f_R(p) + (u_R - u_L) = 0,
 *     with f_K the shock (Rankine-Hugoniot) branch for p > p_K and the
 *     rarefaction (isentropic, Riemann-invariant) branch otherwise;
 *   - u* = (u_L + u_R)/2 + (f_R(p*) - f_L(p*))/2;
 *   - the self-similar solution W(x/t) is sampled wave by wave; the right
 *     wave is evaluated as the left wave of the mirror-image problem.
 * Used to pin the oracle on the Sod tube.  Shares no code with the CUDA path.
 */
#include <math.h>

/* f_K(p) and df_K/dp for side K = (rho_k, p_k, c_k). */
static void side_function(double p, double rk, double pk, double gam,
                          double *f, double *df)
{
    double ck = sqrt(gam * pk / rk);
    if (p > pk) {
        /* shock: mass flux from the Rankine-Hugoniot conditions */
        double a = 2.0 / ((gam + 1.0) * rk);
        double b = (gam - 1.0) / (gam + 1.0) * pk;
        double root = sqrt(a / (p + b));
        *f = (p - pk) * root;
        *df = root * (1.0 - 0.5 * (p - pk) / (p + b));
    } else {
        /* rarefaction: u + 2c/(gam-1) constant, p / rho^gam constant */
        double e = (gam - 1.0) / (2.0 * gam);
        *f = 2.0 * ck / (gam - 1.0) * (pow(p / pk, e) - 1.0);
        *df = pow(p / pk, -(gam + 1.0) / (2.0 * gam)) / (rk * ck);
    }
}

double orc_exact_residual(const double *wl, const double *wr, double gam, double p)
{
    double fl, dl, fr, dr;
    side_function(p, wl[0], wl[2], gam, &fl, &dl);
    side_function(p, wr[0], wr[2], gam, &fr, &dr);
    return fl + fr + (wr[1] - wl[1]);
}

/* Star pressure and velocity for wl, wr = (rho, u, p).  Returns 0 on
   success, -1 when the data create a vacuum, -2 without convergence. */
int orc_exact_star(const double *wl, const double *wr, double gam,
                   double *pstar, double *ustar, int *iters)
{
    double cl = sqrt(gam * wl[2] / wl[0]);
    double cr = sqrt(gam * wr[2] / wr[0]);
    double du = wr[1] - wl[1];
    if (2.0 * (cl + cr) / (gam - 1.0) <= du) return -1;
    /* start from the linearised (acoustic) estimate of p*, kept positive */
    double p = 0.5 * (wl[2] + wr[2]) - 0.125 * du * (wl[0] + wr[0]) * (cl + cr);
    if (!(p > 1e-12)) p = 1e-12;
    int n = 0;
    for (;;) {
        double fl, dl, fr, dr;
        side_function(p, wl[0], wl[2], gam, &fl, &dl);
        side_function(p, wr[0], wr[2], gam, &fr, &dr);
        double next = p - (fl + fr + du) / (dl + dr);
        if (!(next > 1e-14)) next = 1e-14;
        double rel = fabs(next - p) / (0.5 * (next + p));
        p = next;
        ++n;
        if (rel < 1e-14) break;   /* quadratic convergence: roundoff-limited */
        if (n >= 200) return -2;
    }
    double fl, dl, fr, dr;
    side_function(p, wl[0], wl[2], gam, &fl, &dl);
    side_function(p, wr[0], wr[2], gam, &fr, &dr);
    *pstar = p;
    *ustar = 0.5 * (wl[1] + wr[1]) + 0.5 * (fr - fl);
    if (iters) *iters = n;
    return 0;
}

/* State at speed s (s <= u*) produced by the left-moving wave of side
   (rk, uk, pk); out = (rho, u, p). */
static void left_wave(double rk, double uk, double pk, double gam,
                      double pm, double um, double s, double *out)
{
    double ck = sqrt(gam * pk / rk);
    if (pm > pk) {
        double ratio = pm / pk;
        double shock = uk - ck * sqrt((gam + 1.0) / (2.0 * gam) * ratio
                                      + (gam - 1.0) / (2.0 * gam));
        if (s <= shock) { out[0] = rk; out[1] = uk; out[2] = pk; return; }
        double mu = (gam - 1.0) / (gam + 1.0);
        out[0] = rk * (ratio + mu) / (mu * ratio + 1.0);
        out[1] = um;
        out[2] = pm;
        return;
    }
    double head = uk - ck;
    double c_star = ck * pow(pm / pk, (gam - 1.0) / (2.0 * gam));
    double tail = um - c_star;
    if (s <= head) { out[0] = rk; out[1] = uk; out[2] = pk; return; }
    if (s >= tail) { out[0] = rk * pow(pm / pk, 1.0 / gam); out[1] = um; out[2] = pm; return; }
    /* inside the fan: u - c = s and u + 2c/(gam-1) = uk + 2ck/(gam-1) */
    double u = 2.0 / (gam + 1.0) * (ck + 0.5 * (gam - 1.0) * uk + s);
    double c = u - s;
    double rho = rk * pow(c / ck, 2.0 / (gam - 1.0));
    out[0] = rho;
    out[1] = u;
    out[2] = pk * pow(rho / rk, gam);
}

void orc_exact_sample(const double *wl, const double *wr, double gam,
                      double pm, double um, double s, double *out)
{
    if (s <= um) {
        left_wave(wl[0], wl[1], wl[2], gam, pm, um, s, out);
        return;
    }
    /* mirror x -> -x: the right wave becomes a left wave */
    left_wave(wr[0], -wr[1], wr[2], gam, pm, -um, -s, out);
    out[1] = -out[1];
}

/* Sample n points x[i] at time t > 0 for a discontinuity at x0. */
int orc_exact_profile(const double *wl, const double *wr, double gam, double x0,
                      double t, const double *x, long n, double *rho, double *u, double *p)
{
    double pm, um;
    int rc = orc_exact_star(wl, wr, gam, &pm, &um, 0);
    if (rc) return rc;
    for (long i = 0; i < n; ++i) {
        double o[3];
        orc_exact_sample(wl, wr, gam, pm, um, (x[i] - x0) / t, o);
        rho[i] = o[0];
        u[i] = o[1];
        p[i] = o[2];
    }
    return 0;
}
