/*
 * lbm_oracle.h -- plain FP64 CPU oracle for the coupled lattice Boltzmann
 * time step of Tanaka & Iber, "Simulation of a Microfluidic Gradient
 * Generator using Lattice Boltzmann Methods" (arXiv 1307.4703).
 *
 * TEST INFRASTRUCTURE ONLY.  The test-suite, the smoke check and the CPU
 * baseline leg of the benchmark are the only users.  The CUDA library never
 * includes, links or calls anything here, and this code shares nothing with
 * it (no header, no table, no helper).
 *
 * What it computes (section "Numerical Methods"):
 *   fluid   D2Q9 lattice BGK, Eq. lattice / Eq. lbequation / Eq. moments,
 *           f_eq = rho w_i [1 + 3 e.u + 9/2 (e.u)^2 - 3/2 u^2],
 *           nu = c_s^2 (tau_f - 1/2), c_s^2 = 1/3.
 *   scalar  MDF lattice BGK on the four axis directions plus a rest
 *           population of weight w0 (Eq. cdeequilibrium).  w0 = 0 is the
 *           paper's D2Q4 lattice exactly: g_eq = C/4 [1 + 2 e.u],
 *           D = (2 tau_g - 1)/4.  w0 = 1/3 is the common D2Q5 lattice.
 *           In general w_{1..4} = (1-w0)/4, c_s^2 = (1-w0)/2,
 *           g_eq_i = w_i C [1 + e_i.u / c_s^2], D = c_s^2 (tau_g - 1/2).
 *           The velocity u is the fluid velocity of the same node and time.
 *   walls   halfway bounce-back of both lattices (zero flux).
 *   ports   valve-controlled openings on a column: an open velocity port is
 *           a Zou-He velocity node for f and a Dirichlet node C = C_in for
 *           g; an open pressure port is a Zou-He pressure node for f and a
 *           do-nothing node for g (the missing population keeps its own
 *           post-collision value of the previous step, the zeroth-order
 *           extrapolation in time of section "Boundary Conditions").  A
 *           closed port is a wall (section "Results": closed valves are an
 *           ordinary no-flux wall).
 *           The paper's own port boundary (section "Boundary Conditions") is
 *           kept as two more kinds: the unknown populations of f keep the
 *           node's own post-collision values of the previous step
 *           (do-nothing), then all nine are rescaled by
 *           gamma = rho_port / sum f_i to the prescribed density, which
 *           leaves u unchanged.  ORC_PRESSURE_RESCALE is an outlet (g:
 *           do-nothing); ORC_INLET_RESCALE is an inlet whose scalar is set
 *           the same way: do-nothing for the unknown g, then all five are
 *           rescaled to C_in.  When the node holds no compound (sum g = 0)
 *           there is nothing to rescale, and the five take the equilibrium
 *           g_eq(C_in, u) instead.
 *   decay   the reaction term R = -k C of Eq. cde (the decaying compound of
 *           section "Results"), added to the scalar collision as w_i R, so
 *           that the step removes k C from the node's concentration.
 *
 * Populations are stored per node, f[(y*nx + x)*9 + i], g[(y*nx + x)*5 + i],
 * and are the PRE-collision values f_i(x, t) of Eq. lbequation.
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_WEST = 0, ORC_EAST = 1 };
enum { ORC_VELOCITY = 0, ORC_PRESSURE = 1, ORC_PRESSURE_RESCALE = 2, ORC_INLET_RESCALE = 3 };

/* One valve-controlled opening.  It covers the nodes (x, y) for
 * y0 <= y < y1.  WEST: fluid enters or leaves towards -x, so the populations
 * with e_x = +1 are unknown at the node; EAST: the mirror image.  The port is
 * open during a step when bit `channel` of that step's valve word is set. */
typedef struct {
    int channel;
    int side;      /* ORC_WEST or ORC_EAST */
    int x;         /* node column */
    int y0, y1;    /* rows [y0, y1) */
    int kind;      /* ORC_VELOCITY, ORC_PRESSURE, ORC_PRESSURE_RESCALE, ORC_INLET_RESCALE */
    double rho;    /* prescribed density of a pressure port (kinds 1-3) */
} orc_port;

typedef struct orc_lattice orc_lattice;

/* solid: ny*nx bytes, non-zero = solid.  edge_u / edge_C: 2*ny values,
 * [side*ny + y] = u_x and C_in at the velocity-port node of that side and
 * row (ignored elsewhere; may be NULL when there are no velocity ports).
 * periodic != 0 wraps both axes (used only by closed-form checks).
 * Returns NULL on invalid arguments.  The lattice starts at rest:
 * rho = 1, u = 0, C = 0. */
orc_lattice* orc_new(int nx, int ny, const unsigned char* solid,
                     double tau_f, double tau_g, double w0, int periodic,
                     int n_ports, const orc_port* ports,
                     const double* edge_u, const double* edge_C);
void orc_free(orc_lattice* L);

/* Decay rate k >= 0 of the compound (default 0). */
void orc_set_decay(orc_lattice* L, double k);

/* Fluid wall scheme: 0 halfway bounce-back (default); 1 the paper's
 * equilibrium interpolation ("Boundary Conditions"): a population missing at
 * a fluid node because its source is not fluid becomes the equilibrium of a
 * density extrapolated to first order from the fluid along its direction
 * and a momentum interpolated between zero at the wall (half a link behind
 * the node) and the next fluid node.  The scalar keeps bounce-back (zero
 * flux).  Returns 0, or -1 for an unknown scheme or no memory. */
int orc_set_wall_scheme(orc_lattice* L, int scheme);

/* Set every fluid node to the equilibrium of the given fields (ny*nx). */
void orc_init_equilibrium(orc_lattice* L, const double* rho, const double* ux,
                          const double* uy, const double* C);

/* Advance one time step with the given valve word. */
void orc_step(orc_lattice* L, unsigned open_mask);

/* Moments of the current state (Eq. moments; C = sum of g).  Solid nodes
 * report 0.  Any pointer may be NULL. */
void orc_fields(const orc_lattice* L, double* rho, double* ux, double* uy,
                double* C);

/* Pre-collision populations, node-major layout described above. */
void orc_get_populations(const orc_lattice* L, double* f, double* g);
void orc_set_populations(orc_lattice* L, const double* f, const double* g);

/* Post-collision populations of the current state (the right-hand side of
 * Eq. lbequation), node-major, solid nodes 0. */
void orc_post_collision(const orc_lattice* L, double* f, double* g);

/* out[0] = sum rho over fluid nodes, out[1] = sum C over fluid nodes,
 * out[2] = sum rho*u_x and out[3] = sum C*u_x over the nodes of the
 * outlet ports (kinds ORC_PRESSURE and ORC_PRESSURE_RESCALE) that are open
 * under open_mask. */
void orc_diagnostics(const orc_lattice* L, unsigned open_mask, double out[4]);

/* Lattice tables as the oracle uses them (for checks against Eq. lattice). */
void orc_lattice_vectors(int ex[9], int ey[9], double w[9]);

/* Host threads the row loops use: 1 in the serial build
 * (liblbm_oracle.so), the OpenMP team size in the all-cores build of the
 * same source (liblbm_oracle_omp.so).  Both builds give the same bits. */
int orc_num_threads(void);
void orc_set_num_threads(int n);   /* no effect in the serial build */

/* Scalar-only step with a given velocity field (section "Results": the
 * stationary velocity fields are computed once and the advection-diffusion
 * solver reads them; the fluid populations do not change).  ux, uy: ny*nx
 * values already scaled to the scalar's time step.  Same scalar boundary
 * nodes as orc_step. */
void orc_scalar_step(orc_lattice* L, unsigned open_mask, const double* ux, const double* uy);

/* ---- Adjoint (reverse-mode derivative of the time step) ----
 *
 * The step maps the pre-collision state S_t = (f, g) to S_{t+1}; its
 * parameters are tau_g, the inlet velocities u_in (edge_u) and the held
 * concentrations C_in (edge_C).  orc_adjoint_step takes the adjoint of
 * S_{t+1} (af, ag: d J / d S_{t+1}, node-major like the populations) and
 * replaces it, in place, by the adjoint of S_t, given S_t and S_{t+1} and the
 * step's valve word.  It adds the step's parameter derivatives to grad:
 * grad[0] += dJ/d(1/tau_g), grad[1 + side*ny + y] += dJ/du_in(side, y),
 * grad[1 + 2*ny + side*ny + y] += dJ/dC_in(side, y). */
void orc_adjoint_step(const orc_lattice* L, unsigned open_mask, const double* f_t,
                      const double* g_t, const double* f_t1, const double* g_t1,
                      double* af, double* ag, double* grad);

/* Adjoint of lattices whose ports are of kinds ORC_VELOCITY and
 * ORC_PRESSURE, without decay and with bounce-back walls (orc_adjoint
 * returns -1 otherwise).
 * Run n steps forward from the current state with the given valve words
 * (the lattice ends at S_n, as after n calls of orc_step), then the reverse
 * pass for J = sum_k weight_k (C(x_k, y_k, n) - target_k)^2.  Returns J and
 * writes dJ/dtau_g, dJ/du_in (2*ny) and dJ/dC_in (2*ny).  Keeps every state
 * of the trajectory in host memory (test sizes).  Returns a negative value
 * and writes nothing if memory runs out. */
double orc_adjoint(orc_lattice* L, int n, const unsigned* masks, int n_obj,
                   const int* obj_x, const int* obj_y, const double* target,
                   const double* weight, double* dJ_dtau_g, double* dJ_du_in,
                   double* dJ_dC_in);

#ifdef __cplusplus
}
#endif
#endif
