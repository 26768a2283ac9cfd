/*
 * riemann_exact.c -- exact solution of the 1-D Riemann problem for the Euler
 * equations of an ideal gas, used to check the shock-tube runs (Sec. VI: the
 * paper compares with the analytic solution of Sod's problem but does not
 * print it).
 *
 * TEST INFRASTRUCTURE: part of the oracle; only tests, the smoke check and the
 * benchmark's CPU-baseline leg load it.
 *
 * Equation of state: P = rho T (Eq. e with P = (2/D) rho e_t), so the sound
 * speed is c = sqrt(gamma P / rho) with gamma = (D+n+2)/(D+n).
 *
 * Method (the standard exact solver): the star-region pressure p* is the root
 * of f_L(p) + f_R(p) + (u_R - u_L) = 0, where f_K is the shock (Rankine-
 * Hugoniot) branch for p > p_K and the isentropic rarefaction branch for
 * p <= p_K; it is found by Newton iteration.  The solution is then sampled on
 * the self-similar variable S = (x - x0)/t through the wave pattern.
 */
#include <math.h>

typedef struct {
    double rho, u, p, c;
} rstate;

/* f_K(p) and its derivative for one side */
static void pressure_fn(double p, const rstate *K, double g, double *f, double *df)
{
    if (p > K->p) { /* shock */
        double A = 2.0 / ((g + 1.0) * K->rho);
        double B = (g - 1.0) / (g + 1.0) * K->p;
        double q = sqrt(A / (p + B));
        *f = (p - K->p) * q;
        *df = q * (1.0 - 0.5 * (p - K->p) / (p + B));
    } else { /* rarefaction */
        double e = (g - 1.0) / (2.0 * g);
        *f = 2.0 * K->c / (g - 1.0) * (pow(p / K->p, e) - 1.0);
        *df = 1.0 / (K->rho * K->c) * pow(p / K->p, -(g + 1.0) / (2.0 * g));
    }
}

/* star pressure and velocity */
static int star_region(const rstate *L, const rstate *R, double g, double *ps, double *us)
{
    double du = R->u - L->u;
    /* positivity (no vacuum generated) */
    if (2.0 * (L->c + R->c) / (g - 1.0) <= du) return -1;
    /* two-rarefaction estimate as the starting point */
    double e = (g - 1.0) / (2.0 * g);
    double p = pow((L->c + R->c - 0.5 * (g - 1.0) * du) /
                       (L->c / pow(L->p, e) + R->c / pow(R->p, e)),
                   1.0 / e);
    if (!(p > 0.0)) p = 1e-8;
    for (int it = 0; it < 200; ++it) {
        double fL, dL, fR, dR;
        pressure_fn(p, L, g, &fL, &dL);
        pressure_fn(p, R, g, &fR, &dR);
        double pn = p - (fL + fR + du) / (dL + dR);
        if (pn <= 0.0) pn = 0.5 * p;
        double change = fabs(pn - p) / (0.5 * (pn + p));
        p = pn;
        if (change < 1e-15) break;
    }
    double fL, dL, fR, dR;
    pressure_fn(p, L, g, &fL, &dL);
    pressure_fn(p, R, g, &fR, &dR);
    *ps = p;
    *us = 0.5 * (L->u + R->u) + 0.5 * (fR - fL);
    return 0;
}

/* the solution at S = x/t */
static void sample(double S, const rstate *L, const rstate *R, double g, double ps,
                   double us, double *rho, double *u, double *p)
{
    double gm = (g - 1.0) / (g + 1.0);
    if (S <= us) { /* left of the contact */
        if (ps > L->p) { /* left shock */
            double SL = L->u - L->c * sqrt((g + 1.0) / (2.0 * g) * ps / L->p +
                                           (g - 1.0) / (2.0 * g));
            if (S <= SL) { *rho = L->rho; *u = L->u; *p = L->p; }
            else {
                *rho = L->rho * (ps / L->p + gm) / (gm * ps / L->p + 1.0);
                *u = us; *p = ps;
            }
        } else { /* left rarefaction */
            double SH = L->u - L->c;
            double cs = L->c * pow(ps / L->p, (g - 1.0) / (2.0 * g));
            double ST = us - cs;
            if (S <= SH) { *rho = L->rho; *u = L->u; *p = L->p; }
            else if (S > ST) {
                *rho = L->rho * pow(ps / L->p, 1.0 / g); *u = us; *p = ps;
            } else { /* inside the fan */
                double c = 2.0 / (g + 1.0) * (L->c + 0.5 * (g - 1.0) * (L->u - S));
                *u = 2.0 / (g + 1.0) * (L->c + 0.5 * (g - 1.0) * L->u + S);
                *rho = L->rho * pow(c / L->c, 2.0 / (g - 1.0));
                *p = L->p * pow(c / L->c, 2.0 * g / (g - 1.0));
            }
        }
    } else { /* right of the contact */
        if (ps > R->p) { /* right shock */
            double SR = R->u + R->c * sqrt((g + 1.0) / (2.0 * g) * ps / R->p +
                                           (g - 1.0) / (2.0 * g));
            if (S >= SR) { *rho = R->rho; *u = R->u; *p = R->p; }
            else {
                *rho = R->rho * (ps / R->p + gm) / (gm * ps / R->p + 1.0);
                *u = us; *p = ps;
            }
        } else { /* right rarefaction */
            double SH = R->u + R->c;
            double cs = R->c * pow(ps / R->p, (g - 1.0) / (2.0 * g));
            double ST = us + cs;
            if (S >= SH) { *rho = R->rho; *u = R->u; *p = R->p; }
            else if (S < ST) {
                *rho = R->rho * pow(ps / R->p, 1.0 / g); *u = us; *p = ps;
            } else {
                double c = 2.0 / (g + 1.0) * (R->c - 0.5 * (g - 1.0) * (R->u - S));
                *u = 2.0 / (g + 1.0) * (-R->c + 0.5 * (g - 1.0) * R->u + S);
                *rho = R->rho * pow(c / R->c, 2.0 / (g - 1.0));
                *p = R->p * pow(c / R->c, 2.0 * g / (g - 1.0));
            }
        }
    }
}

/* left/right = {rho, u, p}; samples npts points x[] at time t with the
 * diaphragm at x0; star = {p*, u*}.  Returns 0, or -1 for a vacuum. */
int orc_riemann(double gamma, const double *left, const double *right, double x0,
                double t, int npts, const double *x, double *rho, double *u, double *p,
                double *star)
{
    rstate L = {left[0], left[1], left[2], sqrt(gamma * left[2] / left[0])};
    rstate R = {right[0], right[1], right[2], sqrt(gamma * right[2] / right[0])};
    double ps, us;
    if (star_region(&L, &R, gamma, &ps, &us)) return -1;
    star[0] = ps;
    star[1] = us;
    for (int k = 0; k < npts; ++k) {
        double S = (t > 0.0) ? (x[k] - x0) / t : (x[k] < x0 ? -INFINITY : INFINITY);
        sample(S, &L, &R, gamma, ps, us, &rho[k], &u[k], &p[k]);
    }
    return 0;
}
