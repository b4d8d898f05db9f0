/*
 * pflbm_oracle3d.h -- plain FP64 CPU oracle of the three-dimensional form of
 * the scheme (arXiv 2312.00369): D3Q19 for the hydrodynamic lattice (Eq. 3ci
 * and its weights), D3Q7 for the phase lattice (c_s^2 = 1/4, Sec. 2.1.3), the
 * 27-neighbour ghost average of Sec. 2.2.2 (b = 27, c' = [M N]).
 *
 * TEST INFRASTRUCTURE, like pflbm_oracle.h: loaded only by the tests, the
 * smoke check and the CPU legs of the benchmark; it shares nothing with the
 * CUDA path.
 *
 * Nodes are stored [nz][ny][nx], index (z*ny + y)*nx + x. x and y are
 * periodic; z is periodic only with wrap_z (otherwise planes 0, 1, nz-2 and
 * nz-1 must be solid). Velocity orders:
 *   D3Q19: rest; +x, -x, +y, -y, +z, -z; then the 12 edges
 *          (+x+y, -x-y, +x-y, -x+y, +x+z, -x-z, +x-z, -x+z, +y+z, -y-z, +y-z, -y+z);
 *   D3Q7:  the columns of the paper's matrix: rest, +x, -x, +y, -y, +z, -z.
 */
#ifndef PFLBM_ORACLE3D_H
#define PFLBM_ORACLE3D_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct or3_solver or3_solver;

/* D3Q19 (c[19][3], w[19]) and D3Q7 (c[7][3], w[7]) as used here. */
void or3_lattices(int c19[19][3], double w19[19], int c7[7][3], double w7[7]);

/* single-node pieces (pinned by their moments) */
void or3_feq(double p, double rho, const double u[3], double feq[19]);
void or3_geq(double phi, double mu, double alpha, double geq[7]);
void or3_force(double tau_f, const double u[3], const double drho[3], const double F[3], double Fi[19]);
void or3_source(double s, double Gi[7]);
void or3_velocity_pressure(const double f[19], double rho, const double drho[3], const double F[3],
                           double u[3], double* p);
/* isotropic gradient and Laplacian (D3Q19 weights) of a 3x3x3 patch v[dz+1][dy+1][dx+1] */
void or3_stencil(const double v[3][3][3], double g[3], double* lap);

or3_solver* or3_create(int nx, int ny, int nz, int wrap_z, const uint8_t* solid, double theta_deg,
                       double sigma, double W, double M, double tau_f, double rho_l, double rho_g,
                       double tau_g);
void or3_destroy(or3_solver* s);
void or3_params(const or3_solver* s, double out[4]);  /* beta, kappa, tau_g, alpha */
void or3_geometry(const or3_solver* s, uint8_t* cls, double* av);
void or3_init_droplet(or3_solver* s, double x0, double y0, double z0, double R);
void or3_init_phi(or3_solver* s, const double* phi);
/* The (1/2) dG_i/dt term of the phase equation, as in 2D: 0 = backward
 * difference (1/2)[G_i(t) - G_i(t-1)] (default), 1 = omitted. */
void or3_set_dgdt(or3_solver* s, int mode);
void or3_step(or3_solver* s, long n);
/* phi [N], u [N][3], p [N]; any may be NULL */
void or3_get(or3_solver* s, double* phi, double* u, double* p);
double or3_mass(const or3_solver* s);
void or3_budget(const or3_solver* s, double out[4]);

/* Wall for the contact-angle fit. type 0: the plane through p with unit
 * normal n pointing into the fluid; type 1: a solid sphere of centre p and
 * radius r. Only crossings with x_lo <= x < x_hi, y_lo <= y < y_hi and farther
 * than `exclude` from the wall are fitted. */
typedef struct {
    int type;
    double p[3], n[3], r;
    double x_lo, x_hi, y_lo, y_hi;
    double exclude;
} or3_wall_t;

/* Sphere fit (algebraic start, Gauss-Newton on the geometric distance) of the
 * phi = 1/2 crossings between fluid neighbours, and the contact angle: plane
 * cos(theta) = -n.(c - p)/R; sphere cos(theta) = (R^2 + r^2 - D^2)/(2 R r),
 * D = |c - p| (the angle between the two spherical surfaces, measured through
 * the liquid). Returns the number of points; theta is NaN below 4. */
int or3_contact_angle(const double* phi, const uint8_t* cls, int nx, int ny, int nz, const or3_wall_t* wall,
                      double* theta_deg, double sphere[4]);
/* The flat wall z = zw with normal +z. */
int or3_contact_angle_flat(const double* phi, const uint8_t* cls, int nx, int ny, int nz, double zw,
                           double exclude, double* theta_deg, double sphere[4]);

#ifdef __cplusplus
}
#endif
#endif
