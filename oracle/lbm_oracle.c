/*
 * lbm_oracle.c -- plain FP64 CPU oracle for the decoupled Hermite-expansion
 * lattice Boltzmann scheme of Hu, Zhang & Geng, "A decoupled scheme based on
 * the Hermite expansion to construct lattice Boltzmann models for the
 * compressible Navier-Stokes equations with arbitrary specific heat ratio"
 * (arXiv 1606.06107).
 *
 * TEST INFRASTRUCTURE.  This is the slow, obviously-correct reference that the
 * CUDA library is checked against.  Only the test suite, the package smoke
 * check and the benchmark's CPU-baseline leg load it.  It shares no code,
 * header, table or constant generator with the CUDA path: the lattice weights
 * and scaling factor are re-solved here by their own Newton iteration.
 *
 * Everything is double precision and written as straightforward loops over
 * nodes and populations.  Population arrays are population-major, x fastest:
 * a[i*N + (z*Y + y)*X + x], N = X*Y*Z, with no padding.
 *
 * Notation (paper -> here):
 *   g_i (translational populations, Eq. DisEvolI)   -> ft[i]
 *   h_j (rotational populations, Eq. EvoEtaJ)        -> fr[j]
 *   xi_i = r * e_i, e_i integer                      -> e[i][a]
 *   eta_j = r * (j - 3), j = 0..6 (Table II, D1Q7)
 *   theta = T (dimensionless temperature, Eq. DDF with theta0 = 1)
 *
 * Readings of the paper taken here (the paper is garbled or silent):
 *  - Equilibria: the printed a^(k).H^(k) expressions of Sec. IV are garbled;
 *    the standard 4th-order Hermite projection of the Maxwellian is used
 *    (geq_node below).  The pin is that the lattice moments of geq equal the
 *    Maxwellian's moments up to order 4.
 *  - Table I prints k=4 for the Perm(2r,r) and Perm(3r,r) groups; each has 8
 *    members, which is what makes 37 velocities.
 *  - The printed r and weights carry ~9 digits; they are re-solved in FP64
 *    from the Gauss-Hermite moment equations, starting from the printed values.
 *  - eta is scaled as eta/sqrt(n theta0) so that heq has unit variance at T=1
 *    and the rotational energy is e_r = nT/2.
 *  - STREAM mode (the GPU hot path): g is pulled exactly on the lattice with
 *    dt = dx/r (the time mapping of Sec. VI, t = step/(X r)); h is advected by
 *    the fluid velocity with the forward-Euler third-order upwind scheme of
 *    Eq. DisEvolSpaTiJ at Courant number u*dt/dx = u/r.  The stored ft is the
 *    post-collision value, so g_i(x,t) = ft_i(x - e_i).  tau is in lattice
 *    steps: omega = 1/tau.
 *  - FD mode (the paper's literal Eq. DisEvolSpaTiI for g): both g and h by
 *    forward Euler + third-order upwind with dt = dx/(m r), omega = 1/(m tau).
 *  - Step order: moments at time t (Sec. V steps 3-4) from the time-t
 *    populations, then g and h are both updated from time-t values (steps 1-2).
 *  - Boundaries: periodic = wrap; copy (the paper's "open") = clamp the index
 *    to the edge node, applied to the stored arrays.
 *  - Initial state: equilibrium at the given (rho, u, T).  In STREAM mode the
 *    stored ft is the pull pre-image ft_i(y) = geq_i(m0(bc(y + e_i))) so that
 *    the first pull gives g(x,0) = geq(m0(x)) away from clamped edges.
 *  - n = 0: the rotational part has no energy; fr is not stored (Q_r = 0).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_D1Q7 1
#define ORC_D2Q37 2
#define ORC_D2Q49 3
#define ORC_D3Q343 4
#define ORC_QMAX 343

#define ORC_MODE_STREAM 0
#define ORC_MODE_FD 1

#define ORC_BC_PERIODIC 0
#define ORC_BC_COPY 1

typedef struct {
    int kind, D, Q;
    double r;
    int e[ORC_QMAX][3]; /* xi_i = r * e_i */
    double w[ORC_QMAX];
    double resid; /* max |moment residual| after the solve */
} orc_lattice;

/* Simulation description shared with the Python wrapper (plain struct). */
typedef struct {
    int kind;     /* ORC_D1Q7 ... */
    int n;        /* rotational degrees of freedom, gamma = (D+n+2)/(D+n) */
    double tau;   /* relaxation time in lattice steps (STREAM) */
    int mode;     /* ORC_MODE_STREAM or ORC_MODE_FD */
    int m_fd;     /* FD sub-steps per lattice step: dt = dx/(m r) */
    int shape[3]; /* X, Y, Z (unused axes = 1) */
    int bc[3];    /* per axis: ORC_BC_PERIODIC or ORC_BC_COPY */
} orc_cfg;

/* ------------------------------------------------------------------------ */
/* Dense linear solve (Gaussian elimination, partial pivoting), in place.    */
static int solve_dense(int n, double *A, double *b)
{
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(A[r * n + c]) > fabs(A[p * n + c])) p = r;
        if (A[p * n + c] == 0.0) return -1;
        if (p != c) {
            for (int k = 0; k < n; ++k) {
                double t = A[c * n + k]; A[c * n + k] = A[p * n + k]; A[p * n + k] = t;
            }
            double t = b[c]; b[c] = b[p]; b[p] = t;
        }
        for (int r = c + 1; r < n; ++r) {
            double f = A[r * n + c] / A[c * n + c];
            for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
            b[r] -= f * b[c];
        }
    }
    for (int c = n - 1; c >= 0; --c) {
        double s = b[c];
        for (int k = c + 1; k < n; ++k) s -= A[c * n + k] * b[k];
        b[c] = s / A[c * n + c];
    }
    return 0;
}

/* (k-1)!! for even k: the k-th moment of the unit normal distribution. */
static double gauss_moment(int k)
{
    if (k % 2) return 0.0;
    double m = 1.0;
    for (int j = k - 1; j > 1; j -= 2) m *= j;
    return m;
}

/* D1Q7 (Table II): velocities 0, +-r, +-2r, +-3r.  Unknowns w0..w3 and r;
 * equations: the even moments 0,2,4,6,8 of N(0,1) are reproduced exactly. */
static int solve_d1q7(double w[4], double *r_out, double *resid)
{
    double v[5] = {4.766698882e-1, 2.339147370e-1, 2.693818936e-2, 8.121295330e-4,
                   1.1969797752}; /* printed Table II values: the starting point */
    for (int it = 0; it < 100; ++it) {
        double F[5], J[25];
        double r = v[4];
        F[0] = v[0] + 2.0 * (v[1] + v[2] + v[3]) - 1.0;
        J[0] = 1.0; J[1] = 2.0; J[2] = 2.0; J[3] = 2.0; J[4] = 0.0;
        for (int k = 1; k <= 4; ++k) {
            int p = 2 * k;
            double s = 0.0, ds = 0.0;
            J[k * 5 + 0] = 0.0;
            for (int m = 1; m <= 3; ++m) {
                double mp = pow((double)m, p);
                s += 2.0 * v[m] * mp * pow(r, p);
                ds += 2.0 * v[m] * mp * p * pow(r, p - 1);
                J[k * 5 + m] = 2.0 * mp * pow(r, p);
            }
            F[k] = s - gauss_moment(p);
            J[k * 5 + 4] = ds;
        }
        double dv[5];
        for (int k = 0; k < 5; ++k) dv[k] = -F[k];
        if (solve_dense(5, J, dv)) return -1;
        double step = 0.0;
        for (int k = 0; k < 5; ++k) {
            v[k] += dv[k];
            if (fabs(dv[k]) > step) step = fabs(dv[k]);
        }
        if (step < 1e-17) break;
    }
    for (int k = 0; k < 4; ++k) w[k] = v[k];
    *r_out = v[4];
    /* residual of the five equations at the solution */
    double res = fabs(v[0] + 2.0 * (v[1] + v[2] + v[3]) - 1.0);
    for (int k = 1; k <= 4; ++k) {
        double s = 0.0;
        for (int m = 1; m <= 3; ++m) s += 2.0 * v[m] * pow(m * v[4], 2 * k);
        double d = fabs(s - gauss_moment(2 * k)) / gauss_moment(2 * k);
        if (d > res) res = d;
    }
    *resid = res;
    return 0;
}

/* The 8 symmetry groups of D2Q37 (Table I), base vectors in units of r. */
static const int d2q37_base[8][2] = {{0, 0}, {1, 0}, {1, 1}, {2, 0},
                                     {2, 1}, {3, 0}, {3, 1}, {3, 3}};

/* All distinct vectors obtained from (a,b) by sign changes and the swap. */
static int group_members(int a, int b, int out[8][2])
{
    int cand[8][2] = {{a, b}, {-a, b}, {a, -b}, {-a, -b},
                      {b, a}, {-b, a}, {b, -a}, {-b, -a}};
    int n = 0;
    for (int c = 0; c < 8; ++c) {
        int dup = 0;
        for (int k = 0; k < n; ++k)
            if (out[k][0] == cand[c][0] && out[k][1] == cand[c][1]) dup = 1;
        if (!dup) { out[n][0] = cand[c][0]; out[n][1] = cand[c][1]; ++n; }
    }
    return n;
}

/* sum over the members of group g of ex^a * ey^b */
static double group_sum(int g, int a, int b)
{
    int m[8][2];
    int n = group_members(d2q37_base[g][0], d2q37_base[g][1], m);
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += pow((double)m[k][0], a) * pow((double)m[k][1], b);
    return s;
}

/* D2Q37 (Table I): 8 group weights and r from the 9 independent even moment
 * equations of the 2-D unit normal up to degree 8 (odd ones vanish by
 * symmetry, so the quadrature is exact to degree 9). */
static const int d2q37_eq[9][2] = {{0, 0}, {2, 0}, {4, 0}, {2, 2}, {6, 0},
                                   {4, 2}, {8, 0}, {6, 2}, {4, 4}};

static int solve_d2q37(double W[8], double *r_out, double *resid)
{
    double v[9] = {2.03916918e-1, 1.27544846e-1, 4.37537182e-2, 8.13659044e-3,
                   9.40079914e-3, 6.95051049e-4, 3.04298494e-5, 2.81093762e-5,
                   1.1969797752}; /* printed Table I values: the starting point */
    double S[8][9];
    for (int g = 0; g < 8; ++g)
        for (int q = 0; q < 9; ++q) S[g][q] = group_sum(g, d2q37_eq[q][0], d2q37_eq[q][1]);
    for (int it = 0; it < 100; ++it) {
        double F[9], J[81];
        double r = v[8];
        for (int q = 0; q < 9; ++q) {
            int p = d2q37_eq[q][0] + d2q37_eq[q][1];
            double target = gauss_moment(d2q37_eq[q][0]) * gauss_moment(d2q37_eq[q][1]);
            double s = 0.0;
            for (int g = 0; g < 8; ++g) {
                s += v[g] * S[g][q];
                J[q * 9 + g] = pow(r, p) * S[g][q];
            }
            F[q] = pow(r, p) * s - target;
            J[q * 9 + 8] = (p > 0) ? p * pow(r, p - 1) * s : 0.0;
        }
        double dv[9];
        for (int k = 0; k < 9; ++k) dv[k] = -F[k];
        if (solve_dense(9, J, dv)) return -1;
        double step = 0.0;
        for (int k = 0; k < 9; ++k) {
            v[k] += dv[k];
            if (fabs(dv[k]) > step) step = fabs(dv[k]);
        }
        if (step < 1e-17) break;
    }
    for (int g = 0; g < 8; ++g) W[g] = v[g];
    *r_out = v[8];
    double res = 0.0;
    for (int q = 0; q < 9; ++q) {
        int p = d2q37_eq[q][0] + d2q37_eq[q][1];
        double target = gauss_moment(d2q37_eq[q][0]) * gauss_moment(d2q37_eq[q][1]);
        double s = 0.0;
        for (int g = 0; g < 8; ++g) s += v[g] * S[g][q];
        double d = fabs(pow(v[8], p) * s - target) / target;
        if (d > res) res = d;
    }
    *resid = res;
    return 0;
}

/* Order the velocities by (ez, ey, ex) ascending: the population index
 * convention shared (as an interface) with the CUDA library's export. */
static void sort_lattice(orc_lattice *L)
{
    for (int i = 1; i < L->Q; ++i) {
        int e[3] = {L->e[i][0], L->e[i][1], L->e[i][2]};
        double w = L->w[i];
        int k = i - 1;
        while (k >= 0) {
            int *f = L->e[k];
            int gt = (f[2] > e[2]) || (f[2] == e[2] && f[1] > e[1]) ||
                     (f[2] == e[2] && f[1] == e[1] && f[0] > e[0]);
            if (!gt) break;
            memcpy(L->e[k + 1], L->e[k], sizeof(int) * 3);
            L->w[k + 1] = L->w[k];
            --k;
        }
        memcpy(L->e[k + 1], e, sizeof(int) * 3);
        L->w[k + 1] = w;
    }
}

static int build_lattice(int kind, orc_lattice *L)
{
    memset(L, 0, sizeof(*L));
    L->kind = kind;
    double w1[4], r;
    double res1;
    if (solve_d1q7(w1, &r, &res1)) return -1;
    if (kind == ORC_D1Q7) {
        L->D = 1; L->Q = 7; L->r = r; L->resid = res1;
        for (int i = 0; i < 7; ++i) { L->e[i][0] = i - 3; L->w[i] = w1[abs(i - 3)]; }
    } else if (kind == ORC_D2Q49 || kind == ORC_D3Q343) {
        /* tensor products of D1Q7: the D-dimensional unit normal factorises */
        int D = (kind == ORC_D2Q49) ? 2 : 3;
        L->D = D; L->r = r; L->resid = res1;
        int q = 0;
        for (int c = 0; c < (D == 3 ? 7 : 1); ++c)
            for (int b = 0; b < 7; ++b)
                for (int a = 0; a < 7; ++a) {
                    L->e[q][0] = a - 3; L->e[q][1] = b - 3; L->e[q][2] = (D == 3) ? c - 3 : 0;
                    L->w[q] = w1[abs(a - 3)] * w1[abs(b - 3)] * (D == 3 ? w1[abs(c - 3)] : 1.0);
                    ++q;
                }
        L->Q = q;
    } else if (kind == ORC_D2Q37) {
        double W[8], r37, res37;
        if (solve_d2q37(W, &r37, &res37)) return -1;
        L->D = 2; L->r = r37; L->resid = res37;
        int q = 0;
        for (int g = 0; g < 8; ++g) {
            int m[8][2];
            int n = group_members(d2q37_base[g][0], d2q37_base[g][1], m);
            for (int k = 0; k < n; ++k) {
                L->e[q][0] = m[k][0]; L->e[q][1] = m[k][1]; L->e[q][2] = 0;
                L->w[q] = W[g];
                ++q;
            }
        }
        L->Q = q;
    } else {
        return -1;
    }
    sort_lattice(L);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Equilibria (Sec. IV).                                                     */

/* g_i^eq = w_i rho sum_{k<=4} a^(k).H^(k)/k!  -- the 4th-order Hermite
 * projection of the translational Maxwellian g^eq (Eq. DF) with mean u and
 * variance theta, in the reading stated in the file header. */
static void geq_node(const orc_lattice *L, double rho, const double *u, double theta,
                     double *out)
{
    const int D = L->D;
    double u2 = 0.0;
    for (int a = 0; a < D; ++a) u2 += u[a] * u[a];
    double t = theta - 1.0;
    for (int i = 0; i < L->Q; ++i) {
        double c = 0.0, s = 0.0;
        for (int a = 0; a < D; ++a) {
            double xi = L->r * L->e[i][a];
            c += xi * u[a];
            s += xi * xi;
        }
        double h1 = c;
        double h2 = c * c - u2 + t * (s - D);
        double h3 = c * c * c - 3.0 * c * u2 + 3.0 * t * c * (s - D - 2.0);
        double h4 = c * c * c * c - 6.0 * c * c * u2 + 3.0 * u2 * u2 +
                    6.0 * t * (c * c * (s - D - 4.0) + (D + 2.0 - s) * u2) +
                    3.0 * t * t * (s * s - 2.0 * (D + 2.0) * s + D * (D + 2.0));
        out[i] = L->w[i] * rho * (1.0 + h1 + h2 / 2.0 + h3 / 6.0 + h4 / 24.0);
    }
}

/* h_j^eq on D1Q7 (Table II): the same projection in one dimension with zero
 * mean (h^eq has no drift, Eq. DF) and variance theta. */
static void heq_node(const orc_lattice *L1, double theta, double *out)
{
    double t = theta - 1.0;
    for (int j = 0; j < 7; ++j) {
        double eta = L1->r * (j - 3);
        double s = eta * eta;
        out[j] = L1->w[j] * (1.0 + t * (s - 1.0) / 2.0 +
                             t * t * (s * s - 6.0 * s + 3.0) / 8.0);
    }
}

/* Sec. V steps (3)-(4): rho, u and T from the populations at one node.
 * K = sum_i g_i xi_i^2/2 (Eq. TransEnergy), R = sum_j (n/2) h_j eta_j^2
 * (Eq. RotaEnergy), T from Eq. T. */
static void node_moments(const orc_lattice *L, const orc_lattice *L1, int n,
                         const double *g, const double *h, double *rho_o,
                         double *u_o, double *T_o, double *K_o, double *R_o)
{
    const int D = L->D;
    double rho = 0.0, mom[3] = {0, 0, 0}, K = 0.0, R = 0.0;
    for (int i = 0; i < L->Q; ++i) {
        double s = 0.0;
        rho += g[i];
        for (int a = 0; a < D; ++a) {
            double xi = L->r * L->e[i][a];
            mom[a] += g[i] * xi;
            s += xi * xi;
        }
        K += g[i] * 0.5 * s;
    }
    if (n > 0)
        for (int j = 0; j < 7; ++j) {
            double eta = L1->r * (j - 3);
            R += 0.5 * n * h[j] * eta * eta;
        }
    double u2 = 0.0;
    for (int a = 0; a < D; ++a) {
        u_o[a] = mom[a] / rho;
        u2 += u_o[a] * u_o[a];
    }
    *rho_o = rho;
    *T_o = 2.0 / (D + n) * (K + rho * R - 0.5 * rho * u2) / rho;
    if (K_o) *K_o = K;
    if (R_o) *R_o = R;
}

/* ------------------------------------------------------------------------ */
/* Grid helpers.                                                             */

static int bc_index(int x, int X, int bc)
{
    if (bc == ORC_BC_PERIODIC) return ((x % X) + X) % X;
    return x < 0 ? 0 : (x >= X ? X - 1 : x);
}

static long node_of(const orc_cfg *c, int x, int y, int z)
{
    int X = c->shape[0], Y = c->shape[1], Z = c->shape[2];
    x = bc_index(x, X, c->bc[0]);
    y = bc_index(y, Y, c->bc[1]);
    z = bc_index(z, Z, c->bc[2]);
    return ((long)z * Y + y) * X + x;
}

/* Third-order upwind convection term nu * dF/dx along one axis (Sec. V,
 * the stencils under Eq. DisEvolSpaTiI and Eq. DisEvolSpaTiJ), with the
 * Courant number nu = velocity * dt/dx.  F(k) = F at offset k on the axis. */
static double upwind_term(double nu, double Fm2, double Fm1, double F0, double Fp1,
                          double Fp2)
{
    double nu_plus = 0.5 * (nu + fabs(nu));
    double nu_minus = 0.5 * (nu - fabs(nu));
    double back = (Fm2 - 6.0 * Fm1 + 3.0 * F0 + 2.0 * Fp1) / 6.0;
    double fwd = (-Fp2 + 6.0 * Fp1 - 3.0 * F0 - 2.0 * Fm1) / 6.0;
    return nu_plus * back + nu_minus * fwd;
}

/* sum over the D axes of the upwind convection of array F (one population)
 * at node (x,y,z) with per-axis Courant numbers nu[a] */
static double convect(const orc_cfg *c, int D, const double *F, int x, int y, int z,
                      const double *nu)
{
    double acc = 0.0;
    for (int a = 0; a < D; ++a) {
        double v[5];
        for (int k = -2; k <= 2; ++k) {
            int p[3] = {x, y, z};
            p[a] += k;
            v[k + 2] = F[node_of(c, p[0], p[1], p[2])];
        }
        acc += upwind_term(nu[a], v[0], v[1], v[2], v[3], v[4]);
    }
    return acc;
}

static int qr_of(const orc_cfg *c) { return c->n > 0 ? 7 : 0; }

static long nodes_of(const orc_cfg *c)
{
    return (long)c->shape[0] * c->shape[1] * c->shape[2];
}

/* gather the time-t populations g_i(x,t), h_j(x,t) at one node */
static void gather_node(const orc_cfg *c, const orc_lattice *L, const double *ft,
                        const double *fr, int x, int y, int z, double *g, double *h)
{
    long N = nodes_of(c);
    long self = node_of(c, x, y, z);
    for (int i = 0; i < L->Q; ++i) {
        long src = self;
        if (c->mode == ORC_MODE_STREAM) /* pull: g_i(x,t) = ft_i(x - e_i) */
            src = node_of(c, x - L->e[i][0], y - L->e[i][1], z - L->e[i][2]);
        g[i] = ft[i * N + src];
    }
    for (int j = 0; j < qr_of(c); ++j) h[j] = fr[j * N + self];
}

/* ------------------------------------------------------------------------ */
/* Public API (called through ctypes).                                       */

int orc_lattice_get(int kind, double *r, int *e, double *w, double *resid)
{
    orc_lattice L;
    if (build_lattice(kind, &L)) return -1;
    *r = L.r;
    for (int i = 0; i < L.Q; ++i) {
        for (int a = 0; a < 3; ++a) e[i * 3 + a] = L.e[i][a];
        w[i] = L.w[i];
    }
    if (resid) *resid = L.resid;
    return L.Q;
}

int orc_geq(int kind, double rho, const double *u, double theta, double *out)
{
    orc_lattice L;
    if (build_lattice(kind, &L)) return -1;
    geq_node(&L, rho, u, theta, out);
    return L.Q;
}

int orc_heq(double theta, double *out)
{
    orc_lattice L1;
    if (build_lattice(ORC_D1Q7, &L1)) return -1;
    heq_node(&L1, theta, out);
    return 7;
}

/* moments of a single node's populations (Sec. V steps 3-4); out = rho,u[D],T,K,R */
int orc_node_moments(int kind, int n, const double *g, const double *h, double *out)
{
    orc_lattice L, L1;
    if (build_lattice(kind, &L) || build_lattice(ORC_D1Q7, &L1)) return -1;
    double rho, u[3], T, K, R;
    node_moments(&L, &L1, n, g, h, &rho, u, &T, &K, &R);
    out[0] = rho;
    for (int a = 0; a < L.D; ++a) out[1 + a] = u[a];
    out[1 + L.D] = T;
    out[2 + L.D] = K;
    out[3 + L.D] = R;
    return 0;
}

/* BGK relaxation of one node's populations toward the equilibria of its own
 * moments (the collision terms of Eq. DisEvolI / EvoEtaJ), no transport. */
int orc_collide_node(int kind, int n, double omega, const double *g, const double *h,
                     double *g_out, double *h_out)
{
    orc_lattice L, L1;
    if (build_lattice(kind, &L) || build_lattice(ORC_D1Q7, &L1)) return -1;
    double rho, u[3], T, geq[ORC_QMAX], heq[7];
    node_moments(&L, &L1, n, g, h, &rho, u, &T, NULL, NULL);
    geq_node(&L, rho, u, T, geq);
    heq_node(&L1, T, heq);
    for (int i = 0; i < L.Q; ++i) g_out[i] = g[i] - omega * (g[i] - geq[i]);
    if (n > 0)
        for (int j = 0; j < 7; ++j) h_out[j] = h[j] - omega * (h[j] - heq[j]);
    return 0;
}

/* the third-order upwind convection term for one point: f5 = F at offsets
 * -2..+2 along the axis, nu the Courant number (Sec. V) */
double orc_upwind(double nu, const double *f5)
{
    return upwind_term(nu, f5[0], f5[1], f5[2], f5[3], f5[4]);
}

static int check_cfg(const orc_cfg *c, orc_lattice *L, orc_lattice *L1)
{
    if (build_lattice(c->kind, L) || build_lattice(ORC_D1Q7, L1)) return -1;
    for (int a = 0; a < 3; ++a)
        if (c->shape[a] < 1) return -2;
    for (int a = L->D; a < 3; ++a)
        if (c->shape[a] != 1) return -2;
    if (c->n < 0 || !(c->tau > 0.0)) return -1;
    if (c->mode == ORC_MODE_FD && c->m_fd < 1) return -1;
    return 0;
}

/* Initial state: equilibrium at (rho, u, T); u is SoA u[a*N + node]. */
int orc_init(const orc_cfg *c, const double *rho, const double *u, const double *T,
             double *ft, double *fr)
{
    orc_lattice L, L1;
    int rc = check_cfg(c, &L, &L1);
    if (rc) return rc;
    const long N = nodes_of(c);
    const int D = L.D;
    const int X = c->shape[0], Y = c->shape[1], Z = c->shape[2];
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < Z; ++z)
        for (int y = 0; y < Y; ++y)
            for (int x = 0; x < X; ++x) {
                long self = ((long)z * Y + y) * X + x;
                double geq[ORC_QMAX], heq[7];
                for (int i = 0; i < L.Q; ++i) {
                    long src = self;
                    if (c->mode == ORC_MODE_STREAM)
                        src = node_of(c, x + L.e[i][0], y + L.e[i][1], z + L.e[i][2]);
                    double us[3] = {0, 0, 0};
                    for (int a = 0; a < D; ++a) us[a] = u[a * N + src];
                    geq_node(&L, rho[src], us, T[src], geq);
                    ft[i * N + self] = geq[i];
                }
                if (c->n > 0) {
                    heq_node(&L1, T[self], heq);
                    for (int j = 0; j < 7; ++j) fr[j * N + self] = heq[j];
                }
            }
    return 0;
}

/* One time step (Sec. V, steps 1-5 in the reading of the header). */
int orc_step(const orc_cfg *c, const double *ft, const double *fr, double *ft_out,
             double *fr_out)
{
    orc_lattice L, L1;
    int rc = check_cfg(c, &L, &L1);
    if (rc) return rc;
    const long N = nodes_of(c);
    const int D = L.D;
    const int X = c->shape[0], Y = c->shape[1], Z = c->shape[2];
    const int fd = (c->mode == ORC_MODE_FD);
    const double omega = fd ? 1.0 / (c->m_fd * c->tau) : 1.0 / c->tau;
    const double dt_over_dx = fd ? 1.0 / (c->m_fd * L.r) : 1.0 / L.r;
    const int Qr = qr_of(c);
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < Z; ++z)
        for (int y = 0; y < Y; ++y)
            for (int x = 0; x < X; ++x) {
                long self = ((long)z * Y + y) * X + x;
                double g[ORC_QMAX], h[7], geq[ORC_QMAX], heq[7];
                double rho, u[3] = {0, 0, 0}, T;
                gather_node(c, &L, ft, fr, x, y, z, g, h);
                node_moments(&L, &L1, c->n, g, h, &rho, u, &T, NULL, NULL);
                geq_node(&L, rho, u, T, geq);
                for (int i = 0; i < L.Q; ++i) {
                    double out = g[i] - omega * (g[i] - geq[i]);
                    if (fd) { /* Eq. DisEvolSpaTiI: - dt xi_i . grad g_i */
                        double nu[3];
                        for (int a = 0; a < D; ++a) nu[a] = L.r * L.e[i][a] * dt_over_dx;
                        out -= convect(c, D, ft + i * N, x, y, z, nu);
                    }
                    ft_out[i * N + self] = out;
                }
                if (Qr) { /* Eq. DisEvolSpaTiJ: h advected by the fluid velocity u */
                    double nu[3];
                    for (int a = 0; a < D; ++a) nu[a] = u[a] * dt_over_dx;
                    heq_node(&L1, T, heq);
                    for (int j = 0; j < 7; ++j)
                        fr_out[j * N + self] = h[j] - convect(c, D, fr + j * N, x, y, z, nu) -
                                               omega * (h[j] - heq[j]);
                }
            }
    return 0;
}

/* k steps, ping-ponging between (ft, fr) and the scratch pair (ft2, fr2);
 * the result is left in (ft, fr). */
int orc_run(const orc_cfg *c, double *ft, double *fr, double *ft2, double *fr2, long k)
{
    const long N = nodes_of(c);
    orc_lattice L, L1;
    int rc = check_cfg(c, &L, &L1);
    if (rc) return rc;
    for (long s = 0; s < k; ++s) {
        const double *a = (s % 2 == 0) ? ft : ft2;
        const double *b = (s % 2 == 0) ? fr : fr2;
        double *ao = (s % 2 == 0) ? ft2 : ft;
        double *bo = (s % 2 == 0) ? fr2 : fr;
        rc = orc_step(c, a, b, ao, bo);
        if (rc) return rc;
    }
    if (k % 2) {
        memcpy(ft, ft2, sizeof(double) * N * L.Q);
        if (qr_of(c)) memcpy(fr, fr2, sizeof(double) * N * 7);
    }
    return 0;
}

/* rho, u (SoA u[a*N+node]) and T of the current state at every node */
int orc_moments(const orc_cfg *c, const double *ft, const double *fr, double *rho,
                double *u, double *T)
{
    orc_lattice L, L1;
    int rc = check_cfg(c, &L, &L1);
    if (rc) return rc;
    const long N = nodes_of(c);
    const int X = c->shape[0], Y = c->shape[1], Z = c->shape[2];
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < Z; ++z)
        for (int y = 0; y < Y; ++y)
            for (int x = 0; x < X; ++x) {
                long self = ((long)z * Y + y) * X + x;
                double g[ORC_QMAX], h[7], uu[3];
                gather_node(c, &L, ft, fr, x, y, z, g, h);
                node_moments(&L, &L1, c->n, g, h, &rho[self], uu, &T[self], NULL, NULL);
                for (int a = 0; a < L.D; ++a) u[a * N + self] = uu[a];
            }
    return 0;
}

/* Global sums: out = [sum rho, sum rho u_a (D), sum (K + rho R),
 * max_x |sum_j h_j - 1|].  K + rho R = rho (E + u^2/2) is the total energy
 * density of Eq. Total.  Serial loop: a fixed summation order. */
int orc_conservation(const orc_cfg *c, const double *ft, const double *fr, double *out)
{
    orc_lattice L, L1;
    int rc = check_cfg(c, &L, &L1);
    if (rc) return rc;
    const int D = L.D;
    const int X = c->shape[0], Y = c->shape[1], Z = c->shape[2];
    double mass = 0.0, mom[3] = {0, 0, 0}, energy = 0.0, hdev = 0.0;
    for (int z = 0; z < Z; ++z)
        for (int y = 0; y < Y; ++y)
            for (int x = 0; x < X; ++x) {
                double g[ORC_QMAX], h[7], rho, u[3], T, K, R;
                gather_node(c, &L, ft, fr, x, y, z, g, h);
                node_moments(&L, &L1, c->n, g, h, &rho, u, &T, &K, &R);
                mass += rho;
                for (int a = 0; a < D; ++a) mom[a] += rho * u[a];
                energy += K + rho * R;
                if (c->n > 0) {
                    double s = 0.0;
                    for (int j = 0; j < 7; ++j) s += h[j];
                    if (fabs(s - 1.0) > hdev) hdev = fabs(s - 1.0);
                }
            }
    out[0] = mass;
    for (int a = 0; a < D; ++a) out[1 + a] = mom[a];
    out[1 + D] = energy;
    out[2 + D] = hdev;
    return 0;
}
