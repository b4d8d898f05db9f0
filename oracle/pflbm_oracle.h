/*
 * pflbm_oracle.h -- plain FP64 CPU oracle of the phase-field lattice Boltzmann
 * scheme of arXiv 2312.00369 (Ju, Guo, Yan, Sun), in which the liquid-solid
 * surface free energy is folded into the chemical potential (Eq.
 * chemical_potencial2) instead of being imposed as a wetting boundary condition.
 *
 * TEST INFRASTRUCTURE. This library exists to check the CUDA path. Only the
 * test suite, the smoke check and the CPU-baseline / reference legs of the
 * benchmark load it; the product library never links, loads or calls it, and
 * it shares no source, header, table or helper with the CUDA path.
 *
 * Conventions (all lattice units, dx = dt = c = 1):
 *   - nodes are stored row-major, index = y*nx + x; x is always periodic,
 *     y is periodic only when wrap_y != 0 (otherwise a neighbour outside
 *     0..ny-1 does not exist);
 *   - velocity order is the paper's (Eq. ci): c_0=(0,0), c_1..4 =
 *     (cos((i-2)pi/2), sin((i-2)pi/2)), c_5..8 = sqrt2 (cos((i-5)pi/2+pi/4), ...);
 *   - the stored populations f_i, g_i are the post-streaming values (the
 *     state at the start of a time step).
 *
 * Each function is pinned by the tests against the paper's definitions; the
 * readings where the paper is silent (ghost value, doubly-unknown bounce-back,
 * the (1/2) dG/dt history) are pinned by hand-worked values.
 */
#ifndef PFLBM_ORACLE_H
#define PFLBM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Node classes (Sec. 2.2.2-2.2.3). */
enum { OR_FLUID = 0, OR_BOUNDARY = 1, OR_GHOST = 2, OR_INTERIOR = 3 };

typedef struct or_solver or_solver;

/* Lattice of Eq. ci and its weights (Sec. 2.1.2): cx, cy, w, opposite. */
void or_lattice(int cx[9], int cy[9], double w[9], int opp[9]);

/* ---- single-node pieces of the scheme (pinned by moment identities) ---- */
/* f_i^eq of Eq. feq_i with s_i(u) of Eq. Siu. */
void or_feq(double p, double rho, double ux, double uy, double feq[9]);
/* g_i^eq of Eq. H_i (first use of the label, Sec. 2.1.3). */
void or_geq(double phi, double mu, double alpha, double geq[9]);
/* Forcing distribution F_i of Eq. GGi, prefactor (1 - 1/(2 tau_f)). */
void or_force(double tau_f, double ux, double uy, double drx, double dry,
              double Fx, double Fy, double Fi[9]);
/* CH source G_i of Eq. F_i for s = u.grad(phi). */
void or_source(double s, double Gi[9]);
/* Velocity and pressure of Sec. 2.1.2 from f and the force terms. */
void or_velocity_pressure(const double f[9], double rho, double drx, double dry,
                          double Fx, double Fy, double* ux, double* uy, double* p);
/* Isotropic gradient (Eq. gradient) and Laplacian (Eq. Laplace) of a 3x3
 * patch v[dy+1][dx+1]. */
void or_stencil(const double v[3][3], double* gx, double* gy, double* lap);

/* ---- whole-domain solver ---- */
/* Returns NULL on invalid arguments. theta_field_deg may be NULL (uniform
 * theta_deg). tau_g <= 0 selects the default 1.0. When wrap_y == 0 rows 0, 1,
 * ny-2 and ny-1 must be solid. */
or_solver* or_create(int nx, int ny, int wrap_y, const uint8_t* solid,
                     double theta_deg, const double* theta_field_deg,
                     double sigma, double W, double M, double tau_f,
                     double rho_l, double rho_g, double tau_g);
void or_destroy(or_solver* s);
/* Variable viscosity nu(phi) = phi (nu_l - nu_g) + nu_g (both > 0; else the
 * uniform tau_f of or_create) and a body acceleration g (F_b = rho g). */
void or_set_viscosity(or_solver* s, double nu_l, double nu_g);
void or_set_body_force(or_solver* s, double gx, double gy);
/* Treatment of (1/2) dt^2 dG_i/dt in Eq. BGK: 0 backward difference
 * (default, reading R4), 1 omitted (source G_i(t) only). */
void or_set_dgdt(or_solver* s, int mode);
/* Appendix A, Table 2: chi_case 2 (default) is the paper's method; 1 and 3
 * move the wall energy into a Robin ghost condition on flat walls. */
void or_set_chi_case(or_solver* s, int chi_case);
/* Derived parameters: beta, kappa, tau_g, alpha (see or_create). */
void or_params(const or_solver* s, double out[4]);
/* Geometry: class per node, the paper's zeta, epsilon and a_v, and the
 * unknown-link mask (bit i set when zeta(x - c_i) = 0 at a zeta=1 node, paper
 * order) and the doubly-unknown mask (also zeta(x + c_i) = 0). Any may be NULL. */
void or_geometry(const or_solver* s, uint8_t* cls, uint8_t* zeta, double* eps,
                 double* av, uint16_t* unknown, uint16_t* doubly);
/* Initial droplet, Eq. initialphi. The first call after create or after a step
 * replaces phi; later calls keep the pointwise maximum. */
void or_init_droplet(or_solver* s, double x0, double y0, double R);
/* Eq. initialphi at one point, with the x-periodic distance of period
 * nx_period (0: no wrap). */
double or_droplet_phi(double x, double y, double x0, double y0, double R, double W, int nx_period);
/* The same at n points; out[k] = max(out[k], phi) when combine != 0. */
void or_droplet_phi_points(const double* x, const double* y, long n, double x0, double y0,
                           double R, double W, int nx_period, int combine, double* out);
/* General initial field (values on zeta=1 nodes are used). */
void or_init_phi(or_solver* s, const double* phi);
/* n time steps. */
void or_step(or_solver* s, long n);
/* Macroscopic fields of the current state; any pointer may be NULL.
 * u is interleaved (ux, uy) per node. */
void or_get(or_solver* s, double* phi, double* u, double* p);
/* FP64 sum of phi = sum_i g_i over zeta=1 nodes. */
double or_mass(const or_solver* s);
/* Budget of the last step: out = {mass before, source sum, streamed into
 * zeta=0, bounce-back assigned}; mass after = out0 + out1 - out2 + out3. */
void or_budget(const or_solver* s, double out[4]);
/* Raw state access for tests: f, g as [9][ny*nx] in paper order, s_prev. */
void or_state(const or_solver* s, double* f, double* g, double* s_prev);
/* Raw state for tests: overwrite the post-streaming f and g ([9][ny*nx], paper
 * order). The u.grad(phi) history and whether a step has been taken are kept,
 * so a hand-set state can be stepped as the first or as a later step. */
void or_set_state(or_solver* s, const double* f, const double* g);
long or_steps(const or_solver* s);

/* ---- contact-angle measurement (a reading; the paper does not say how) ---- */
/* wall type 0: straight wall through (px, py) with unit normal (nx_, ny_)
 * pointing into the fluid. type 1: circular solid of centre (px, py), radius r.
 * Crossing points of phi = 1/2 between FLUID neighbours at a distance larger
 * than `exclude` from the wall and with x_lo <= x < x_hi are fitted with a
 * circle (algebraic fit, then Gauss-Newton on the geometric distance).
 * Returns the number of points used (< 3: failure). circle = {a, b, R}. */
typedef struct {
    int type;
    double px, py, nx_, ny_, r;
    double x_lo, x_hi;
    double exclude;
} or_wall;
int or_contact_angle(const double* phi, const uint8_t* cls, int nx, int ny,
                     const or_wall* wall, double* theta_deg, double circle[3]);
/* Circle fit alone (points as x[k], y[k]). Returns 0 on success. */
int or_circle_fit(const double* x, const double* y, int n, double circle[3]);

#ifdef __cplusplus
}
#endif
#endif
