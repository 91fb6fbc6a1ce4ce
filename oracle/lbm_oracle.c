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
                 (P->kind == ORC_VELOCITY || P->kind == ORC_PRESSURE);
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
    free(L);
}

void orc_init_equilibrium(orc_lattice* L, const double* rho, const double* ux,
                          const double* uy, const double* C)
{
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
            for (int i = 0; i < 5; ++i)
                gp[c * 5 + i] = gn[i] - (gn[i] - geq(L, i, C, ux, uy)) / L->tau_g;
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

    /* 1. collision (moments of Eq. moments, relaxation of Eq. lbequation) */
    collide_all(L, L->fp, L->gp);

    /* 2. free flight f_i(x + e_i, t + 1) = f_i^post(x, t).  A link that ends
     *    outside the fluid (solid node, outside the domain, or a port's
     *    ghost column) is a wall: the population returns to x with the
     *    opposite direction (halfway bounce-back, zero flux).  Every
     *    population of every fluid node is written exactly once here. */
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
            } else {
                zou_he(fn, s, ORC_PRESSURE, 0.0, P->rho);
                /* do-nothing: zeroth-order extrapolation in time */
                gn[g_in] = L->gp[c * 5 + g_in];
            }
        }
    }
}

void orc_fields(const orc_lattice* L, double* rho, double* ux, double* uy,
                double* C)
{
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
        if (P->kind != ORC_PRESSURE || !((open_mask >> P->channel) & 1u))
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
