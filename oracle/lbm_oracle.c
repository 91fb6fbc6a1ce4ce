/*
 * lbm_oracle.c -- plain FP64 CPU oracle of the coupled D2Q9 + scalar lattice
 * Boltzmann step (Tanaka & Iber, arXiv 1307.4703, "Numerical Methods" and
 * "Boundary Conditions").
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the CPU
 * baseline of the benchmark; never by the CUDA library, with which it shares
 * no code.
 *
 * The code follows the paper's two-step reading of Eq. lbequation: at every
 * fluid node the populations relax towards the local equilibrium
 * (collision), then every population flies to the neighbouring node
 * x + e_i (free flight); boundary nodes are completed afterwards.  It is
 * written for clarity, not speed: one full copy of the post-collision
 * populations, dense loops, no fusion.
 */
#include "lbm_oracle.h"

#include <stdlib.h>
#include <string.h>

/* Row loops whose iterations write disjoint memory (every destination value
 * has exactly one writer) run on all host cores in the OpenMP build of this
 * file (liblbm_oracle_omp.so).  Each value is computed by the same
 * expression in either build, so both give the same bits.  Sums over the
 * lattice (diagnostics, the adjoint's parameter derivatives) stay serial. */
#ifdef _OPENMP
#include <omp.h>
#define ORC_ROWS _Pragma("omp parallel for schedule(static)")
#else
#define ORC_ROWS
#endif

/* Eq. lattice: i = 0 rest; i = 1..4 the axis directions at angles
 * pi (i-1)/2 (east, north, west, south); i = 5..8 the diagonals at angles
 * pi (i - 9/2)/2 with length sqrt(2) (north-east, north-west, south-west,
 * south-east). */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
/* index of -e_i */
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
/* D2Q9 weights (the w_i equation of "Numerical Methods") */
static const double W9[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                             1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

struct orc_lattice {
    int nx, ny, periodic;
    double tau_f, tau_g, w0;
    double decay;          /* k of the reaction term R = -k C */
    int wall_scheme;       /* 0 halfway bounce-back, 1 equilibrium interpolation */
    double* mom;           /* rho, j_x, j_y of every node at the start of a step (scheme 1) */
    unsigned char* solid;  /* ny*nx */
    double* f;             /* pre-collision f_i(x,t), [node*9 + i] */
    double* g;             /* pre-collision g_i(x,t), [node*5 + i] */
    double* fp;            /* post-collision copies (work arrays) */
    double* gp;
    int n_ports;
    orc_port* ports;
    double* edge_u;        /* [side*ny + y] */
    double* edge_C;
};

static int node(const orc_lattice* L, int x, int y) { return y * L->nx + x; }

static int is_fluid(const orc_lattice* L, int x, int y)
{
    if (x < 0 || x >= L->nx || y < 0 || y >= L->ny) return 0;
    return L->solid[node(L, x, y)] == 0;
}

/* f_eq of the D2Q9 BGK equation ("Numerical Methods"). */
static double feq(int i, double rho, double ux, double uy)
{
    double eu = EX[i] * ux + EY[i] * uy;
    double uu = ux * ux + uy * uy;
    return rho * W9[i] * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
}

/* Scalar lattice weight: rest weight w0, the four axis directions share
 * the rest equally.  w0 = 0 gives the paper's 1/4 (Eq. cdeequilibrium). */
static double wg(const orc_lattice* L, int i)
{
    return i == 0 ? L->w0 : 0.25 * (1.0 - L->w0);
}

/* Scalar equilibrium g_eq_i = w_i C [1 + e_i.u / c_s^2],
 * c_s^2 = (1 - w0)/2; for w0 = 0 this is C/4 [1 + 2 e_i.u]. */
static double geq(const orc_lattice* L, int i, double C, double ux, double uy)
{
    double cs2 = 0.5 * (1.0 - L->w0);
    double eu = EX[i] * ux + EY[i] * uy;
    return wg(L, i) * C * (1.0 + eu / cs2);
}

/* Eq. moments (the sum runs over the nine populations i = 0..8). */
static void moments(const double* fn, double* rho, double* ux, double* uy)
{
    double r = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < 9; ++i) {
        r += fn[i];
        jx += fn[i] * EX[i];
        jy += fn[i] * EY[i];
    }
    *rho = r;
    *ux = jx / r;
    *uy = jy / r;
}

static double scalar_moment(const double* gn)
{
    double C = 0.0;
    for (int i = 0; i < 5; ++i) C += gn[i];
    return C;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

void orc_lattice_vectors(int ex[9], int ey[9], double w[9])
{
    for (int i = 0; i < 9; ++i) {
        ex[i] = EX[i];
        ey[i] = EY[i];
        w[i] = W9[i];
    }
}

orc_lattice* orc_new(int nx, int ny, const unsigned char* solid,
                     double tau_f, double tau_g, double w0, int periodic,
                     int n_ports, const orc_port* ports,
                     const double* edge_u, const double* edge_C)
{
    if (nx < 1 || ny < 1 || !solid || !(tau_f > 0.5) || !(tau_g > 0.5))
        return NULL;
    if (!(w0 >= 0.0 && w0 < 1.0) || n_ports < 0 || (n_ports > 0 && !ports))
        return NULL;
    orc_lattice* L = (orc_lattice*)calloc(1, sizeof(orc_lattice));
    if (!L) return NULL;
    size_t n = (size_t)nx * (size_t)ny;
    L->nx = nx;
    L->ny = ny;
    L->periodic = periodic;
    L->tau_f = tau_f;
    L->tau_g = tau_g;
    L->w0 = w0;
    L->solid = (unsigned char*)malloc(n);
    L->f = (double*)calloc(n * 9, sizeof(double));
    L->g = (double*)calloc(n * 5, sizeof(double));
    L->fp = (double*)calloc(n * 9, sizeof(double));
    L->gp = (double*)calloc(n * 5, sizeof(double));
    L->edge_u = (double*)calloc(2 * (size_t)ny, sizeof(double));
    L->edge_C = (double*)calloc(2 * (size_t)ny, sizeof(double));
    L->ports = (orc_port*)calloc(n_ports > 0 ? (size_t)n_ports : 1,
                                 sizeof(orc_port));
    if (!L->solid || !L->f || !L->g || !L->fp || !L->gp || !L->edge_u ||
        !L->edge_C || !L->ports) {
        orc_free(L);
        return NULL;
    }
    for (size_t k = 0; k < n; ++k) L->solid[k] = solid[k] ? 1 : 0;
    L->n_ports = n_ports;
    for (int p = 0; p < n_ports; ++p) {
        const orc_port* P = &ports[p];
        int ok = P->channel >= 0 && P->channel < 32 && P->x >= 0 &&
                 P->x < nx && P->y0 >= 0 && P->y0 < P->y1 && P->y1 <= ny &&
                 (P->side == ORC_WEST || P->side == ORC_EAST) &&
                 P->kind >= ORC_VELOCITY && P->kind <= ORC_INLET_RESCALE &&
                 (P->kind == ORC_VELOCITY || P->rho > 0.0);
        for (int y = P->y0; ok && y < P->y1; ++y)
            ok = L->solid[y * nx + P->x] == 0;
        if (!ok) {
            orc_free(L);
            return NULL;
        }
        L->ports[p] = *P;
    }
    if (edge_u) memcpy(L->edge_u, edge_u, 2 * (size_t)ny * sizeof(double));
    if (edge_C) memcpy(L->edge_C, edge_C, 2 * (size_t)ny * sizeof(double));
    /* rest state rho = 1, u = 0, C = 0 */
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            if (!is_fluid(L, x, y)) continue;
            int c = node(L, x, y);
            for (int i = 0; i < 9; ++i) L->f[c * 9 + i] = feq(i, 1.0, 0.0, 0.0);
        }
    return L;
}

void orc_free(orc_lattice* L)
{
    if (!L) return;
    free(L->solid);
    free(L->f);
    free(L->g);
    free(L->fp);
    free(L->gp);
    free(L->edge_u);
    free(L->edge_C);
    free(L->ports);
    free(L->mom);
    free(L);
}

void orc_set_decay(orc_lattice* L, double k) { L->decay = k; }

int orc_set_wall_scheme(orc_lattice* L, int scheme)
{
    if (scheme != 0 && scheme != 1) return -1;
    if (scheme == 1 && !L->mom) {
        L->mom = (double*)calloc((size_t)L->nx * (size_t)L->ny * 3, sizeof(double));
        if (!L->mom) return -1;
    }
    L->wall_scheme = scheme;
    return 0;
}

/* The paper's wall ("Boundary Conditions"): the population f_m missing at
 * fluid node (x, y) -- its source (x, y) - e_m is not fluid -- becomes the
 * equilibrium of a density extrapolated to first order from the fluid in
 * the direction e_m, 2 rho(x + e_m) - rho(x + 2 e_m), and a momentum
 * interpolated linearly between zero at the wall, half a link behind the
 * node, and the fluid node x + e_m one and a half links from it:
 * j = j(x + e_m) / 3.  Moments are those at the start of the step.  Where
 * x + 2 e_m is not fluid the density is that of x + e_m; where x + e_m is
 * not fluid either, the node's own density with zero momentum. */
static double wall_population(const orc_lattice* L, int x, int y, int m)
{
    const double* M = L->mom;
    int x1 = x + EX[m], y1 = y + EY[m], x2 = x + 2 * EX[m], y2 = y + 2 * EY[m];
    if (L->periodic) {
        x1 = (x1 + L->nx) % L->nx;
        y1 = (y1 + L->ny) % L->ny;
        x2 = (x2 + L->nx) % L->nx;
        y2 = (y2 + L->ny) % L->ny;
    }
    double rho, jx = 0.0, jy = 0.0;
    if (is_fluid(L, x1, y1)) {
        const double* m1 = M + (size_t)node(L, x1, y1) * 3;
        rho = is_fluid(L, x2, y2) ? 2.0 * m1[0] - M[(size_t)node(L, x2, y2) * 3] : m1[0];
        jx = m1[1] / 3.0;
        jy = m1[2] / 3.0;
    } else {
        rho = M[(size_t)node(L, x, y) * 3];
    }
    return feq(m, rho, jx / rho, jy / rho);
}

void orc_init_equilibrium(orc_lattice* L, const double* rho, const double* ux,
                          const double* uy, const double* C)
{
    ORC_ROWS
    for (int y = 0; y < L->ny; ++y)
        for (int x = 0; x < L->nx; ++x) {
            if (!is_fluid(L, x, y)) continue;
            int c = node(L, x, y);
            for (int i = 0; i < 9; ++i)
                L->f[c * 9 + i] = feq(i, rho[c], ux[c], uy[c]);
            for (int i = 0; i < 5; ++i)
                L->g[c * 5 + i] = geq(L, i, C[c], ux[c], uy[c]);
        }
}

/* Collision at every fluid node: the right-hand side of Eq. lbequation for
 * f, and its scalar counterpart for g with the fluid velocity of the same
 * node (the velocity "transferred from the fluid solver"). */
static void collide_all(const orc_lattice* L, double* fp, double* gp)
{
    ORC_ROWS
    for (int y = 0; y < L->ny; ++y)
        for (int x = 0; x < L->nx; ++x) {
            if (!is_fluid(L, x, y)) continue;
            int c = node(L, x, y);
            const double* fn = L->f + (size_t)c * 9;
            const double* gn = L->g + (size_t)c * 5;
            double rho, ux, uy;
            moments(fn, &rho, &ux, &uy);
            for (int i = 0; i < 9; ++i)
                fp[c * 9 + i] = fn[i] - (fn[i] - feq(i, rho, ux, uy)) / L->tau_f;
            double C = scalar_moment(gn);
            double R = -L->decay * C;  /* reaction term of Eq. cde */
            for (int i = 0; i < 5; ++i)
                gp[c * 5 + i] = gn[i] - (gn[i] - geq(L, i, C, ux, uy)) / L->tau_g + wg(L, i) * R;
        }
}

/* The paper's port boundary for f (section "Boundary Conditions"): the
 * unknown populations (e_x = s) keep the node's own post-collision values
 * fpn of the previous step, then every population is rescaled by
 * gamma = rho_port / sum f_i. */
static void rescale_port_f(double* fn, const double* fpn, int s, double rho_port)
{
    int unknown[3] = {s > 0 ? 1 : 3, s > 0 ? 5 : 6, s > 0 ? 8 : 7};
    for (int k = 0; k < 3; ++k) fn[unknown[k]] = fpn[unknown[k]];
    double sum = 0.0;
    for (int i = 0; i < 9; ++i) sum += fn[i];
    double gamma = rho_port / sum;
    for (int i = 0; i < 9; ++i) fn[i] *= gamma;
}

/* The same for g at an inlet: do-nothing for the unknown population, then
 * all five rescaled to C_in; with no compound at the node, the equilibrium
 * of C_in at the node's velocity. */
static void rescale_port_g(const orc_lattice* L, double* gn, const double* gpn, int g_in, double C_in,
                           double ux, double uy)
{
    gn[g_in] = gpn[g_in];
    double sum = scalar_moment(gn);
    if (sum > 0.0) {
        double gamma = C_in / sum;
        for (int i = 0; i < 5; ++i) gn[i] *= gamma;
    } else {
        for (int i = 0; i < 5; ++i) gn[i] = geq(L, i, C_in, ux, uy);
    }
}

/* Zou-He completion of the three unknown populations of a port node.  s is
 * +1 on a WEST port (unknowns e_x = +1: 1, 5, 8) and -1 on an EAST port
 * (unknowns 3, 6, 7).  The tangential velocity is zero.  A velocity node
 * takes u_x and solves the density from the known populations; a pressure
 * node takes rho and solves u_x.  The unknowns follow from bounce-back of
 * the non-equilibrium part along the normal and from the momentum balance
 * along the wall (Zou & He 1997). */
static void zou_he(double* fn, int s, int kind, double u_in, double rho_in)
{
    int axis_in = s > 0 ? 1 : 3;      /* e = (s, 0)  */
    int diag_in_up = s > 0 ? 5 : 6;   /* e = (s, +1) */
    int diag_in_dn = s > 0 ? 8 : 7;   /* e = (s, -1) */
    int axis_out = OPP[axis_in];      /* e = (-s, 0)  */
    int diag_out_dn = OPP[diag_in_up];/* e = (-s, -1) */
    int diag_out_up = OPP[diag_in_dn];/* e = (-s, +1) */
    /* rho (1 - s u_x) = f0 + f2 + f4 + 2 (sum of the populations leaving) */
    double K = fn[0] + fn[2] + fn[4] +
               2.0 * (fn[axis_out] + fn[diag_out_dn] + fn[diag_out_up]);
    double rho, ux;
    if (kind == ORC_VELOCITY) {
        ux = u_in;
        rho = K / (1.0 - s * ux);
    } else {
        rho = rho_in;
        ux = s * (1.0 - K / rho);
    }
    double jx = rho * ux;  /* the tangential momentum rho u_y is zero */
    fn[axis_in] = fn[axis_out] + s * (2.0 / 3.0) * jx;
    fn[diag_in_up] = fn[diag_out_dn] - 0.5 * (fn[2] - fn[4]) +
                     s * (1.0 / 6.0) * jx;
    fn[diag_in_dn] = fn[diag_out_up] + 0.5 * (fn[2] - fn[4]) +
                     s * (1.0 / 6.0) * jx;
}

void orc_step(orc_lattice* L, unsigned open_mask)
{
    const int nx = L->nx, ny = L->ny;

    /* moments at the start of the step, for the paper's wall scheme */
    if (L->wall_scheme == 1) {
        ORC_ROWS
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                if (!is_fluid(L, x, y)) continue;
                int c = node(L, x, y);
                double r, ux, uy;
                moments(L->f + (size_t)c * 9, &r, &ux, &uy);
                L->mom[(size_t)c * 3] = r;
                L->mom[(size_t)c * 3 + 1] = r * ux;
                L->mom[(size_t)c * 3 + 2] = r * uy;
            }
    }

    /* 1. collision (moments of Eq. moments, relaxation of Eq. lbequation) */
    collide_all(L, L->fp, L->gp);

    /* 2. free flight f_i(x + e_i, t + 1) = f_i^post(x, t).  A link that ends
     *    outside the fluid (solid node, outside the domain, or a port's
     *    ghost column) is a wall: the population returns to x with the
     *    opposite direction (halfway bounce-back, zero flux).  Every
     *    population of every fluid node is written exactly once here. */
    ORC_ROWS
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            if (!is_fluid(L, x, y)) continue;
            int c = node(L, x, y);
            for (int i = 0; i < 9; ++i) {
                int xn = x + EX[i], yn = y + EY[i];
                if (L->periodic) {
                    xn = (xn + nx) % nx;
                    yn = (yn + ny) % ny;
                }
                if (is_fluid(L, xn, yn))
                    L->f[node(L, xn, yn) * 9 + i] = L->fp[c * 9 + i];
                else if (L->wall_scheme == 1)
                    L->f[c * 9 + OPP[i]] = wall_population(L, x, y, OPP[i]);
                else
                    L->f[c * 9 + OPP[i]] = L->fp[c * 9 + i];
            }
            for (int i = 0; i < 5; ++i) {
                int xn = x + EX[i], yn = y + EY[i];
                if (L->periodic) {
                    xn = (xn + nx) % nx;
                    yn = (yn + ny) % ny;
                }
                if (is_fluid(L, xn, yn))
                    L->g[node(L, xn, yn) * 5 + i] = L->gp[c * 5 + i];
                else
                    L->g[c * 5 + OPP[i]] = L->gp[c * 5 + i];
            }
        }

    /* 3. open valves: inlet and outlet nodes replace the populations that
     *    arrive from outside the domain.  A closed valve keeps the wall of
     *    step 2. */
    for (int p = 0; p < L->n_ports; ++p) {
        const orc_port* P = &L->ports[p];
        if (!((open_mask >> P->channel) & 1u)) continue;
        int s = P->side == ORC_WEST ? 1 : -1;
        int g_in = s > 0 ? 1 : 3;  /* scalar population with e_x = s */
        for (int y = P->y0; y < P->y1; ++y) {
            int c = node(L, P->x, y);
            double* fn = L->f + (size_t)c * 9;
            double* gn = L->g + (size_t)c * 5;
            if (P->kind == ORC_VELOCITY) {
                zou_he(fn, s, ORC_VELOCITY, L->edge_u[P->side * ny + y], 0.0);
                /* prescribed concentration: the unknown population makes
                 * the node's zeroth moment equal C_in */
                double others = 0.0;
                for (int i = 0; i < 5; ++i)
                    if (i != g_in) others += gn[i];
                gn[g_in] = L->edge_C[P->side * ny + y] - others;
            } else if (P->kind == ORC_PRESSURE) {
                zou_he(fn, s, ORC_PRESSURE, 0.0, P->rho);
                /* do-nothing: zeroth-order extrapolation in time */
                gn[g_in] = L->gp[c * 5 + g_in];
            } else {
                rescale_port_f(fn, L->fp + (size_t)c * 9, s, P->rho);
                if (P->kind == ORC_PRESSURE_RESCALE) {
                    gn[g_in] = L->gp[c * 5 + g_in];
                } else {
                    double r, ux, uy;
                    moments(fn, &r, &ux, &uy);
                    rescale_port_g(L, gn, L->gp + (size_t)c * 5, g_in, L->edge_C[P->side * ny + y], ux, uy);
                }
            }
        }
    }
}

void orc_fields(const orc_lattice* L, double* rho, double* ux, double* uy,
                double* C)
{
    ORC_ROWS
    for (int y = 0; y < L->ny; ++y)
        for (int x = 0; x < L->nx; ++x) {
            int c = node(L, x, y);
            double r = 0.0, vx = 0.0, vy = 0.0, cc = 0.0;
            if (is_fluid(L, x, y)) {
                moments(L->f + (size_t)c * 9, &r, &vx, &vy);
                cc = scalar_moment(L->g + (size_t)c * 5);
            }
            if (rho) rho[c] = r;
            if (ux) ux[c] = vx;
            if (uy) uy[c] = vy;
            if (C) C[c] = cc;
        }
}

void orc_get_populations(const orc_lattice* L, double* f, double* g)
{
    size_t n = (size_t)L->nx * (size_t)L->ny;
    if (f) memcpy(f, L->f, n * 9 * sizeof(double));
    if (g) memcpy(g, L->g, n * 5 * sizeof(double));
}

void orc_set_populations(orc_lattice* L, const double* f, const double* g)
{
    size_t n = (size_t)L->nx * (size_t)L->ny;
    if (f) memcpy(L->f, f, n * 9 * sizeof(double));
    if (g) memcpy(L->g, g, n * 5 * sizeof(double));
}

void orc_post_collision(const orc_lattice* L, double* f, double* g)
{
    size_t n = (size_t)L->nx * (size_t)L->ny;
    double* fp = (double*)calloc(n * 9, sizeof(double));
    double* gp = (double*)calloc(n * 5, sizeof(double));
    if (fp && gp) {
        collide_all(L, fp, gp);
        if (f) memcpy(f, fp, n * 9 * sizeof(double));
        if (g) memcpy(g, gp, n * 5 * sizeof(double));
    }
    free(fp);
    free(gp);
}

void orc_diagnostics(const orc_lattice* L, unsigned open_mask, double out[4])
{
    double m = 0.0, mc = 0.0, q = 0.0, qc = 0.0;
    for (int y = 0; y < L->ny; ++y)
        for (int x = 0; x < L->nx; ++x) {
            if (!is_fluid(L, x, y)) continue;
            int c = node(L, x, y);
            double r, ux, uy;
            moments(L->f + (size_t)c * 9, &r, &ux, &uy);
            m += r;
            mc += scalar_moment(L->g + (size_t)c * 5);
        }
    for (int p = 0; p < L->n_ports; ++p) {
        const orc_port* P = &L->ports[p];
        if ((P->kind != ORC_PRESSURE && P->kind != ORC_PRESSURE_RESCALE) || !((open_mask >> P->channel) & 1u))
            continue;
        for (int y = P->y0; y < P->y1; ++y) {
            int c = node(L, P->x, y);
            double r, ux, uy;
            moments(L->f + (size_t)c * 9, &r, &ux, &uy);
            q += r * ux;
            qc += scalar_moment(L->g + (size_t)c * 5) * ux;
        }
    }
    out[0] = m;
    out[1] = mc;
    out[2] = q;
    out[3] = qc;
}

/* ------------------------------------------------------------------------
 * Adjoint of one step (reverse mode).  The forward step is
 *   S_{t+1} = B(P(K(S_t)))
 * with K the collision at every fluid node (Eq. lbequation and its scalar
 * counterpart), P the free flight with bounce-back (a permutation of the
 * post-collision values), B the open-port completion (affine in the values it
 * reads).  The adjoint applies the transposes in reverse order:
 *   a_t = K'(S_t)^T P^T B^T a_{t+1}.
 * ------------------------------------------------------------------------ */

/* Transpose of the Zou-He completion at one node.  kn holds the node's
 * values of S_{t+1} (the known populations are the streamed ones); a is the
 * node's adjoint, whose three unknown entries are folded into the known ones
 * and cleared.  Returns dJ/du_in for a velocity node (0 otherwise). */
static double zou_he_adjoint(const double* kn, double* a, int s, int kind, double u_in, double rho_in)
{
    int axis_in = s > 0 ? 1 : 3;
    int diag_in_up = s > 0 ? 5 : 6;
    int diag_in_dn = s > 0 ? 8 : 7;
    int axis_out = OPP[axis_in];
    int diag_out_dn = OPP[diag_in_up];
    int diag_out_up = OPP[diag_in_dn];
    double a_ax = a[axis_in], a_up = a[diag_in_up], a_dn = a[diag_in_dn];
    a[axis_in] = a[diag_in_up] = a[diag_in_dn] = 0.0;
    /* direct terms: f_ax_in = f_ax_out + ..., f_up = f_dout_dn - (f2 - f4)/2 + ...,
     * f_dn = f_dout_up + (f2 - f4)/2 + ... */
    a[axis_out] += a_ax;
    a[diag_out_dn] += a_up;
    a[diag_out_up] += a_dn;
    a[2] += -0.5 * a_up + 0.5 * a_dn;
    a[4] += 0.5 * a_up - 0.5 * a_dn;
    /* through the node's x momentum jx: dJ/djx */
    double G = s * (2.0 / 3.0) * a_ax + s * (1.0 / 6.0) * (a_up + a_dn);
    double K = kn[0] + kn[2] + kn[4] + 2.0 * (kn[axis_out] + kn[diag_out_dn] + kn[diag_out_up]);
    double dK, du = 0.0;
    if (kind == ORC_VELOCITY) {
        double den = 1.0 - s * u_in;
        dK = G * u_in / den;            /* jx = K u / (1 - s u) */
        du = G * K / (den * den);
    } else {
        (void)rho_in;
        dK = -s * G;                    /* jx = s (rho - K) */
    }
    a[0] += dK;
    a[2] += dK;
    a[4] += dK;
    a[axis_out] += 2.0 * dK;
    a[diag_out_dn] += 2.0 * dK;
    a[diag_out_up] += 2.0 * dK;
    return du;
}

/* Transpose of the collision at one node with pre-collision values fn, gn:
 * on entry af/ag hold the adjoint of the post-collision values, on exit the
 * adjoint of the pre-collision values.  Returns dJ/d(1/tau_g) of the node. */
static double collide_adjoint(const orc_lattice* L, const double* fn, const double* gn, double* af,
                              double* ag)
{
    double rho, ux, uy;
    moments(fn, &rho, &ux, &uy);
    double C = scalar_moment(gn);
    double w = 1.0 / L->tau_f, omg = 1.0 / L->tau_g;
    double cs2 = 0.5 * (1.0 - L->w0);
    double uu = ux * ux + uy * uy;
    /* f_eq_k = w_k [rho + 3 e.j + 9/2 (e.j)^2 / rho - 3/2 j^2 / rho], j = rho u:
     * derivatives with respect to rho (j fixed) and to j */
    double Ar = 0.0, Ax = 0.0, Ay = 0.0;
    for (int k = 0; k < 9; ++k) {
        double eu = EX[k] * ux + EY[k] * uy;
        Ar += af[k] * W9[k] * (1.0 - 4.5 * eu * eu + 1.5 * uu);
        Ax += af[k] * W9[k] * (3.0 * EX[k] + 9.0 * eu * EX[k] - 3.0 * ux);
        Ay += af[k] * W9[k] * (3.0 * EY[k] + 9.0 * eu * EY[k] - 3.0 * uy);
    }
    /* g_eq_k = w_k C [1 + e.j / (rho c_s^2)]: derivatives with respect to C,
     * rho and j */
    double Bc = 0.0, Br = 0.0, Bx = 0.0, By = 0.0, dwg = 0.0;
    for (int k = 0; k < 5; ++k) {
        double eu = EX[k] * ux + EY[k] * uy;
        double wk = wg(L, k);
        Bc += ag[k] * wk * (1.0 + eu / cs2);
        Br += ag[k] * wk * C * (-eu / (rho * cs2));
        Bx += ag[k] * wk * C * EX[k] / (rho * cs2);
        By += ag[k] * wk * C * EY[k] / (rho * cs2);
        dwg += ag[k] * (geq(L, k, C, ux, uy) - gn[k]);
    }
    double nf[9], ng[5];
    for (int i = 0; i < 9; ++i)
        nf[i] = (1.0 - w) * af[i] + w * (Ar + Ax * EX[i] + Ay * EY[i]) +
                omg * (Br + Bx * EX[i] + By * EY[i]);
    for (int i = 0; i < 5; ++i) ng[i] = (1.0 - omg) * ag[i] + omg * Bc;
    for (int i = 0; i < 9; ++i) af[i] = nf[i];
    for (int i = 0; i < 5; ++i) ag[i] = ng[i];
    return dwg;
}

void orc_adjoint_step(const orc_lattice* L, unsigned open_mask, const double* f_t,
                      const double* g_t, const double* f_t1, const double* g_t1,
                      double* af, double* ag, double* grad)
{
    const int nx = L->nx, ny = L->ny;
    size_t n = (size_t)nx * (size_t)ny;
    double* bf = (double*)calloc(n * 9, sizeof(double)); /* adjoint after B^T */
    double* dn = (double*)calloc(n, sizeof(double));     /* do-nothing terms */
    double* pf = (double*)calloc(n * 9, sizeof(double)); /* adjoint of post-collision */
    double* pg = (double*)calloc(n * 5, sizeof(double));
    if (!bf || !dn || !pf || !pg) {
        free(bf); free(dn); free(pf); free(pg);
        return;
    }
    (void)g_t1;
    /* B^T: fold the adjoint of every completed (unknown) population into the
     * populations it was computed from */
    for (int p = 0; p < L->n_ports; ++p) {
        const orc_port* P = &L->ports[p];
        if (!((open_mask >> P->channel) & 1u)) continue;
        int s = P->side == ORC_WEST ? 1 : -1;
        int g_in = s > 0 ? 1 : 3;
        for (int y = P->y0; y < P->y1; ++y) {
            int c = node(L, P->x, y);
            double* a = af + (size_t)c * 9;
            double* b = ag + (size_t)c * 5;
            if (P->kind == ORC_VELOCITY) {
                grad[1 + P->side * ny + y] +=
                    zou_he_adjoint(f_t1 + (size_t)c * 9, a, s, ORC_VELOCITY, L->edge_u[P->side * ny + y], 0.0);
                /* g_in = C_in - sum of the others */
                double ain = b[g_in];
                b[g_in] = 0.0;
                for (int i = 0; i < 5; ++i)
                    if (i != g_in) b[i] -= ain;
                grad[1 + 2 * ny + P->side * ny + y] += ain;
            } else {
                zou_he_adjoint(f_t1 + (size_t)c * 9, a, s, ORC_PRESSURE, 0.0, P->rho);
                /* g_in(t+1) = its own post-collision value at t */
                dn[c] = b[g_in];
                b[g_in] = 0.0;
            }
        }
    }
    memcpy(bf, af, n * 9 * sizeof(double));
    /* P^T: every post-collision value went to exactly one place */
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            if (!is_fluid(L, x, y)) continue;
            int c = node(L, x, y);
            for (int i = 0; i < 9; ++i) {
                int xn = x + EX[i], yn = y + EY[i];
                if (L->periodic) {
                    xn = (xn + nx) % nx;
                    yn = (yn + ny) % ny;
                }
                if (is_fluid(L, xn, yn)) pf[c * 9 + i] = bf[node(L, xn, yn) * 9 + i];
                else pf[c * 9 + i] = bf[c * 9 + OPP[i]];
            }
            for (int i = 0; i < 5; ++i) {
                int xn = x + EX[i], yn = y + EY[i];
                if (L->periodic) {
                    xn = (xn + nx) % nx;
                    yn = (yn + ny) % ny;
                }
                if (is_fluid(L, xn, yn)) pg[c * 5 + i] = ag[node(L, xn, yn) * 5 + i];
                else pg[c * 5 + i] = ag[c * 5 + OPP[i]];
            }
        }
    for (int p = 0; p < L->n_ports; ++p) {
        const orc_port* P = &L->ports[p];
        if (P->kind != ORC_PRESSURE || !((open_mask >> P->channel) & 1u)) continue;
        int g_in = P->side == ORC_WEST ? 1 : 3;
        for (int y = P->y0; y < P->y1; ++y) {
            int c = node(L, P->x, y);
            pg[c * 5 + g_in] += dn[c];
        }
    }
    /* K^T at every fluid node, with the pre-collision values of S_t */
    memset(af, 0, n * 9 * sizeof(double));
    memset(ag, 0, n * 5 * sizeof(double));
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            if (!is_fluid(L, x, y)) continue;
            int c = node(L, x, y);
            double* a = pf + (size_t)c * 9;
            double* b = pg + (size_t)c * 5;
            grad[0] += collide_adjoint(L, f_t + (size_t)c * 9, g_t + (size_t)c * 5, a, b);
            memcpy(af + (size_t)c * 9, a, 9 * sizeof(double));
            memcpy(ag + (size_t)c * 5, b, 5 * sizeof(double));
        }
    free(bf);
    free(dn);
    free(pf);
    free(pg);
}

double orc_adjoint(orc_lattice* L, int n, const unsigned* masks, int n_obj,
                   const int* obj_x, const int* obj_y, const double* target,
                   const double* weight, double* dJ_dtau_g, double* dJ_du_in,
                   double* dJ_dC_in)
{
    const int ny = L->ny;
    if (L->decay != 0.0 || L->wall_scheme != 0) return -1.0;
    for (int p = 0; p < L->n_ports; ++p)
        if (L->ports[p].kind != ORC_VELOCITY && L->ports[p].kind != ORC_PRESSURE) return -1.0;
    size_t nodes = (size_t)L->nx * (size_t)ny;
    double* fs = (double*)malloc((size_t)(n + 1) * nodes * 9 * sizeof(double));
    double* gs = (double*)malloc((size_t)(n + 1) * nodes * 5 * sizeof(double));
    double* af = (double*)calloc(nodes * 9, sizeof(double));
    double* ag = (double*)calloc(nodes * 5, sizeof(double));
    double* grad = (double*)calloc(1 + 4 * (size_t)ny, sizeof(double));
    if (!fs || !gs || !af || !ag || !grad) {
        free(fs); free(gs); free(af); free(ag); free(grad);
        return -1.0;
    }
    memcpy(fs, L->f, nodes * 9 * sizeof(double));
    memcpy(gs, L->g, nodes * 5 * sizeof(double));
    for (int t = 0; t < n; ++t) {
        orc_step(L, masks[t]);
        memcpy(fs + (size_t)(t + 1) * nodes * 9, L->f, nodes * 9 * sizeof(double));
        memcpy(gs + (size_t)(t + 1) * nodes * 5, L->g, nodes * 5 * sizeof(double));
    }
    /* J and its derivative with respect to S_n: C = sum of g */
    double J = 0.0;
    for (int k = 0; k < n_obj; ++k) {
        int c = node(L, obj_x[k], obj_y[k]);
        double C = scalar_moment(L->g + (size_t)c * 5);
        double d = C - target[k];
        J += weight[k] * d * d;
        for (int i = 0; i < 5; ++i) ag[(size_t)c * 5 + i] += 2.0 * weight[k] * d;
    }
    for (int t = n - 1; t >= 0; --t)
        orc_adjoint_step(L, masks[t], fs + (size_t)t * nodes * 9, gs + (size_t)t * nodes * 5,
                         fs + (size_t)(t + 1) * nodes * 9, gs + (size_t)(t + 1) * nodes * 5, af, ag, grad);
    /* d(1/tau_g)/dtau_g = -1/tau_g^2 */
    *dJ_dtau_g = -grad[0] / (L->tau_g * L->tau_g);
    for (int k = 0; k < 2 * ny; ++k) {
        dJ_du_in[k] = grad[1 + k];
        dJ_dC_in[k] = grad[1 + 2 * ny + k];
    }
    free(fs); free(gs); free(af); free(ag); free(grad);
    return J;
}

void orc_scalar_step(orc_lattice* L, unsigned open_mask, const double* ux, const double* uy)
{
    const int nx = L->nx, ny = L->ny;
    /* collision with the given velocity (scalar counterpart of Eq. lbequation
     * with the equilibrium of Eq. cdeequilibrium) */
    ORC_ROWS
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            if (!is_fluid(L, x, y)) continue;
            int c = node(L, x, y);
            const double* gn = L->g + (size_t)c * 5;
            double C = scalar_moment(gn);
            double R = -L->decay * C;  /* reaction term of Eq. cde */
            for (int i = 0; i < 5; ++i)
                L->gp[c * 5 + i] = gn[i] - (gn[i] - geq(L, i, C, ux[c], uy[c])) / L->tau_g + wg(L, i) * R;
        }
    /* free flight with halfway bounce-back */
    ORC_ROWS
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            if (!is_fluid(L, x, y)) continue;
            int c = node(L, x, y);
            for (int i = 0; i < 5; ++i) {
                int xn = x + EX[i], yn = y + EY[i];
                if (L->periodic) {
                    xn = (xn + nx) % nx;
                    yn = (yn + ny) % ny;
                }
                if (is_fluid(L, xn, yn)) L->g[node(L, xn, yn) * 5 + i] = L->gp[c * 5 + i];
                else L->g[c * 5 + OPP[i]] = L->gp[c * 5 + i];
            }
        }
    /* open valves: held concentration at inlets, do-nothing at outlets */
    for (int p = 0; p < L->n_ports; ++p) {
        const orc_port* P = &L->ports[p];
        if (!((open_mask >> P->channel) & 1u)) continue;
        int g_in = P->side == ORC_WEST ? 1 : 3;
        for (int y = P->y0; y < P->y1; ++y) {
            int c = node(L, P->x, y);
            double* gn = L->g + (size_t)c * 5;
            if (P->kind == ORC_VELOCITY) {
                double others = 0.0;
                for (int i = 0; i < 5; ++i)
                    if (i != g_in) others += gn[i];
                gn[g_in] = L->edge_C[P->side * ny + y] - others;
            } else if (P->kind == ORC_INLET_RESCALE) {
                rescale_port_g(L, gn, L->gp + (size_t)c * 5, g_in, L->edge_C[P->side * ny + y], ux[c], uy[c]);
            } else {
                gn[g_in] = L->gp[c * 5 + g_in];
            }
        }
    }
}
