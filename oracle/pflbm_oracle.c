/*
 * pflbm_oracle.c -- plain FP64 CPU oracle of arXiv 2312.00369's phase-field
 * lattice Boltzmann time step (wetting energy inside the chemical potential).
 *
 * TEST INFRASTRUCTURE: see pflbm_oracle.h. Written for a reader checking it
 * against the paper: one loop per step of the algorithm, in the paper's order
 * and notation, no blocking, fusion or reordering.
 *
 * Readings of places where the paper is silent or garbled (each is repeated
 * in the design notes of the repository):
 *   R1 beta = 12 sigma / W, kappa = 3 sigma W / 2: the only pair for which
 *      the tanh profile of Eq. initialphi (width W) solves mu = 0 and
 *      sigma = sqrt(2 kappa beta)/6 (Young's law, Eqs. b1 and sigma_sl).
 *   R2 tau_g defaults to 1 and alpha = M / (c_s^2 (tau_g - 1/2)) (Eq. mobility).
 *   R3 the prefactor of Eq. GGi is (1 - 1/(2 tau_f)) (the printed tau_g can
 *      only be a typo for a force in the f equation).
 *   R4 (1/2) dt dG_i/dt of Eq. BGK is the backward difference
 *      (G_i(t) - G_i(t-1))/2; on the first step the history equals the
 *      current value (zero derivative).
 *   R5 node classes: a solid node with a non-solid 8-neighbour is a boundary
 *      node (zeta = 1, epsilon = 0); a non-solid node is fluid (zeta = 1,
 *      epsilon = 1); a remaining solid node with a zeta = 1 neighbour is a
 *      ghost node (zeta = 0) whose phi is the zeta-weighted mean of its 3x3
 *      neighbourhood; other solid nodes are interior (zeta = 0, phi = 0).
 *   R6 modified bounce-back: an unknown population f_i(x_b) (zeta(x_b - c_i)
 *      = 0) takes the post-streaming f_{i'}(x_b); when that one is unknown too
 *      (zeta(x_b + c_i) = 0) it takes the node's own post-collision f*_{i'}.
 *   R7 initial state: u = 0, p = 0, so f_i = f_i^eq(0, 0) = 0 and
 *      g_i = g_i^eq(phi_0, mu_0).
 *   R9 Appendix A (Table 2) variants on flat walls: the ghost node takes the
 *      value for which the wall-normal difference (phi_b - phi_g) equals
 *      chi(phi_w) = c (phi_w - phi_w^2), phi_w = (phi_b + phi_g)/2, with phi_b
 *      the zeta = 1 node straight above or below it (the normal of a flat
 *      wall points to that node) and c = -sqrt(2 beta/kappa) cos(theta)
 *      (case 1, mu without the a_v term) or +sqrt(2 beta/kappa) cos(theta)
 *      (case 3, mu with twice the a_v term). Case 2 is the paper's method.
 *   R8 body force: F = F_s + F_b with F_b = rho g (a uniform acceleration);
 *      variable viscosity: nu(phi) = phi (nu_l - nu_g) + nu_g (Sec. 2.1.1)
 *      gives tau_f(x) = nu(phi(x)) / c_s^2 + 1/2 (Sec. 2.1.2), used in the
 *      f collision and in the prefactor of Eq. GGi at that node.
 */
#include "pflbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define Q 9
static const double CS2 = 1.0 / 3.0; /* c_s^2 = c^2/3 (D2Q9) */

/* ------------------------------------------------------------------------ */
/* Lattice, Eq. ci and the D2Q9 weights of Sec. 2.1.2.                       */
/* ------------------------------------------------------------------------ */
void or_lattice(int cx[9], int cy[9], double w[9], int opp[9])
{
    cx[0] = 0;
    cy[0] = 0;
    for (int i = 1; i <= 4; ++i) {
        double a = (i - 2) * M_PI / 2.0;
        cx[i] = (int)lround(cos(a));
        cy[i] = (int)lround(sin(a));
    }
    for (int i = 5; i <= 8; ++i) {
        double a = (i - 5) * M_PI / 2.0 + M_PI / 4.0;
        cx[i] = (int)lround(sqrt(2.0) * cos(a));
        cy[i] = (int)lround(sqrt(2.0) * sin(a));
    }
    for (int i = 0; i < Q; ++i) {
        w[i] = (i == 0) ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
    for (int i = 0; i < Q; ++i) {
        opp[i] = -1;
        for (int j = 0; j < Q; ++j) {
            if (cx[j] == -cx[i] && cy[j] == -cy[i]) opp[i] = j;
        }
    }
}

static int CX[Q], CY[Q], OPP[Q];
static double WI[Q];
static int lattice_ready = 0;

static void lattice(void)
{
    if (!lattice_ready) {
        or_lattice(CX, CY, WI, OPP);
        lattice_ready = 1;
    }
}

/* ------------------------------------------------------------------------ */
/* Single-node pieces                                                        */
/* ------------------------------------------------------------------------ */

/* s_i(u), Eq. Siu. */
static double s_i(int i, double ux, double uy)
{
    double cu = CX[i] * ux + CY[i] * uy;
    double uu = ux * ux + uy * uy;
    return WI[i] * (cu / CS2 + (cu * cu) / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}

/* Eq. feq_i. */
void or_feq(double p, double rho, double ux, double uy, double feq[9])
{
    lattice();
    for (int i = 0; i < Q; ++i) {
        if (i == 0)
            feq[i] = p / CS2 * (WI[0] - 1.0) + rho * s_i(0, ux, uy);
        else
            feq[i] = p / CS2 * WI[i] + rho * s_i(i, ux, uy);
    }
}

/* Eq. H_i (Sec. 2.1.3). */
void or_geq(double phi, double mu, double alpha, double geq[9])
{
    lattice();
    geq[0] = phi - (1.0 - WI[0]) * alpha * mu;
    for (int i = 1; i < Q; ++i) geq[i] = WI[i] * alpha * mu;
}

/* Eq. GGi with tau_f in the prefactor (reading R3). The double contraction
 * (u grad rho):(c_i c_i - c_s^2 I) = (c_i.u)(c_i.grad rho) - c_s^2 u.grad rho. */
void or_force(double tau_f, double ux, double uy, double drx, double dry,
              double Fx, double Fy, double Fi[9])
{
    lattice();
    double pre = 1.0 - 1.0 / (2.0 * tau_f);
    double u_grad_rho = ux * drx + uy * dry;
    for (int i = 0; i < Q; ++i) {
        double cF = CX[i] * Fx + CY[i] * Fy;
        double cu = CX[i] * ux + CY[i] * uy;
        double cdr = CX[i] * drx + CY[i] * dry;
        double contraction = cu * cdr - CS2 * u_grad_rho;
        Fi[i] = pre * WI[i] * (u_grad_rho + cF / CS2 + contraction / CS2);
    }
}

/* Eq. F_i (the CH source): I:(c_i c_i - c_s^2 I) = |c_i|^2 - 2 c_s^2 in 2D. */
void or_source(double s, double Gi[9])
{
    lattice();
    for (int i = 0; i < Q; ++i) {
        double c2 = (double)(CX[i] * CX[i] + CY[i] * CY[i]);
        Gi[i] = WI[i] * s * (-1.0 + (c2 - 2.0 * CS2) / (2.0 * CS2));
    }
}

/* Sec. 2.1.2: rho u = sum_i c_i f_i + F/2, then
 * p = c_s^2/(1 - w_0) [sum_{i!=0} f_i + u.grad(rho)/2 + rho s_0(u)]. */
void or_velocity_pressure(const double f[9], double rho, double drx, double dry,
                          double Fx, double Fy, double* ux, double* uy, double* p)
{
    lattice();
    double mx = 0.0, my = 0.0;
    for (int i = 0; i < Q; ++i) {
        mx += CX[i] * f[i];
        my += CY[i] * f[i];
    }
    double vx = (mx + 0.5 * Fx) / rho;
    double vy = (my + 0.5 * Fy) / rho;
    double sum = 0.0;
    for (int i = 1; i < Q; ++i) sum += f[i];
    *p = CS2 / (1.0 - WI[0]) * (sum + 0.5 * (vx * drx + vy * dry) + rho * s_i(0, vx, vy));
    *ux = vx;
    *uy = vy;
}

/* Eqs. gradient and Laplace on a 3x3 patch v[dy+1][dx+1]. */
void or_stencil(const double v[3][3], double* gx, double* gy, double* lap)
{
    lattice();
    double ax = 0.0, ay = 0.0, l = 0.0;
    double v0 = v[1][1];
    for (int i = 1; i < Q; ++i) {
        double vi = v[CY[i] + 1][CX[i] + 1];
        ax += WI[i] * CX[i] * vi / CS2;
        ay += WI[i] * CY[i] * vi / CS2;
        l += 2.0 * WI[i] * (vi - v0) / CS2;
    }
    *gx = ax;
    *gy = ay;
    *lap = l;
}

/* ------------------------------------------------------------------------ */
/* Solver                                                                    */
/* ------------------------------------------------------------------------ */
struct or_solver {
    int nx, ny, wrap_y;
    long N;
    double sigma, W, M, tau_f, tau_g, rho_l, rho_g;
    double beta, kappa, alpha;
    double nu_l, nu_g;   /* > 0: variable viscosity (reading R8) */
    double gx, gy;       /* body acceleration */
    int dgdt;            /* 0: (1/2) dG/dt as a backward difference (R4); 1: omitted */
    int chi_case;        /* Appendix A, Table 2: 1, 2 (default) or 3 (reading R9) */
    uint8_t* cls;
    uint8_t* zeta;
    double* eps;
    double* av;
    double* costh;
    double* f;      /* [Q][N] post-streaming */
    double* g;
    double* fpost;  /* [Q][N] post-collision */
    double* gpost;
    double* s_prev; /* u.grad(phi) of the previous step */
    int history;    /* 0 before the first step (reading R4) */
    int replace_phi;
    double* phi;
    double* mu;
    double* gpx;
    double* gpy;
    double* lap;
    double* ux;
    double* uy;
    double* p;
    double budget[4];
    long steps;
};

/* Neighbour x + (dx, dy); -1 when it leaves the domain in y. */
static long nb(const or_solver* s, int x, int y, int dx, int dy)
{
    int xx = (x + dx) % s->nx;
    if (xx < 0) xx += s->nx;
    int yy = y + dy;
    if (s->wrap_y) {
        yy %= s->ny;
        if (yy < 0) yy += s->ny;
    } else if (yy < 0 || yy >= s->ny) {
        return -1;
    }
    return (long)yy * s->nx + xx;
}

static void* xcalloc(long n, long sz)
{
    return calloc((size_t)(n > 0 ? n : 1), (size_t)sz);
}

/* Sec. 2.2.2 / 2.2.3: classes, zeta, epsilon (Eq. H_i, second use) and
 * a_v = |grad epsilon| with the gradient of Eq. gradient (Eq. avvv). */
static void classify(or_solver* s, const uint8_t* solid)
{
    int nx = s->nx, ny = s->ny;
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            long k = (long)y * nx + x;
            if (!solid[k]) {
                s->cls[k] = OR_FLUID;
                continue;
            }
            int touches_fluid = 0;
            for (int i = 1; i < Q; ++i) {
                long m = nb(s, x, y, CX[i], CY[i]);
                if (m >= 0 && !solid[m]) touches_fluid = 1;
            }
            s->cls[k] = touches_fluid ? OR_BOUNDARY : OR_INTERIOR;
        }
    }
    for (long k = 0; k < s->N; ++k)
        s->zeta[k] = (s->cls[k] == OR_FLUID || s->cls[k] == OR_BOUNDARY) ? 1 : 0;
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            long k = (long)y * nx + x;
            if (s->cls[k] != OR_INTERIOR) continue;
            for (int i = 1; i < Q; ++i) {
                long m = nb(s, x, y, CX[i], CY[i]);
                if (m >= 0 && s->zeta[m]) s->cls[k] = OR_GHOST;
            }
        }
    }
    for (long k = 0; k < s->N; ++k) s->eps[k] = (s->cls[k] == OR_FLUID) ? 1.0 : 0.0;
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            long k = (long)y * nx + x;
            s->av[k] = 0.0;
            if (!s->zeta[k]) continue;
            double v[3][3];
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    long m = nb(s, x, y, dx, dy);
                    v[dy + 1][dx + 1] = (m >= 0) ? s->eps[m] : 0.0;
                }
            double gx, gy, lap;
            or_stencil(v, &gx, &gy, &lap);
            s->av[k] = sqrt(gx * gx + gy * gy);
        }
    }
}

or_solver* or_create(int nx, int ny, int wrap_y, const uint8_t* solid,
                     double theta_deg, const double* theta_field_deg,
                     double sigma, double W, double M, double tau_f,
                     double rho_l, double rho_g, double tau_g)
{
    lattice();
    if (nx < 3 || ny < 3 || !solid || !(sigma >= 0) || !(W > 0) || !(M > 0) ||
        !(tau_f > 0.5) || !(rho_l > 0) || !(rho_g > 0))
        return NULL;
    if (tau_g <= 0) tau_g = 1.0;
    if (!(tau_g > 0.5)) return NULL;
    if (!wrap_y) {
        for (int x = 0; x < nx; ++x) {
            if (!solid[x] || !solid[nx + x] || !solid[(long)(ny - 2) * nx + x] ||
                !solid[(long)(ny - 1) * nx + x])
                return NULL;
        }
    }
    or_solver* s = (or_solver*)calloc(1, sizeof(or_solver));
    s->nx = nx;
    s->ny = ny;
    s->wrap_y = wrap_y ? 1 : 0;
    s->N = (long)nx * ny;
    s->sigma = sigma;
    s->W = W;
    s->M = M;
    s->tau_f = tau_f;
    s->tau_g = tau_g;
    s->rho_l = rho_l;
    s->rho_g = rho_g;
    /* Reading R1. */
    s->beta = 12.0 * sigma / W;
    s->kappa = 3.0 * sigma * W / 2.0;
    /* Reading R2, Eq. mobility: M = c_s^2 alpha (tau_g - 1/2). */
    s->alpha = M / (CS2 * (tau_g - 0.5));

    long N = s->N;
    s->cls = (uint8_t*)xcalloc(N, 1);
    s->zeta = (uint8_t*)xcalloc(N, 1);
    s->eps = (double*)xcalloc(N, sizeof(double));
    s->av = (double*)xcalloc(N, sizeof(double));
    s->costh = (double*)xcalloc(N, sizeof(double));
    s->f = (double*)xcalloc(Q * N, sizeof(double));
    s->g = (double*)xcalloc(Q * N, sizeof(double));
    s->fpost = (double*)xcalloc(Q * N, sizeof(double));
    s->gpost = (double*)xcalloc(Q * N, sizeof(double));
    s->s_prev = (double*)xcalloc(N, sizeof(double));
    s->phi = (double*)xcalloc(N, sizeof(double));
    s->mu = (double*)xcalloc(N, sizeof(double));
    s->gpx = (double*)xcalloc(N, sizeof(double));
    s->gpy = (double*)xcalloc(N, sizeof(double));
    s->lap = (double*)xcalloc(N, sizeof(double));
    s->ux = (double*)xcalloc(N, sizeof(double));
    s->uy = (double*)xcalloc(N, sizeof(double));
    s->p = (double*)xcalloc(N, sizeof(double));
    classify(s, solid);
    for (long k = 0; k < N; ++k) {
        double th = theta_field_deg ? theta_field_deg[k] : theta_deg;
        s->costh[k] = cos(th * M_PI / 180.0);
    }
    s->replace_phi = 1;
    s->chi_case = 2;
    return s;
}

void or_destroy(or_solver* s)
{
    if (!s) return;
    free(s->cls);
    free(s->zeta);
    free(s->eps);
    free(s->av);
    free(s->costh);
    free(s->f);
    free(s->g);
    free(s->fpost);
    free(s->gpost);
    free(s->s_prev);
    free(s->phi);
    free(s->mu);
    free(s->gpx);
    free(s->gpy);
    free(s->lap);
    free(s->ux);
    free(s->uy);
    free(s->p);
    free(s);
}

void or_set_viscosity(or_solver* s, double nu_l, double nu_g)
{
    s->nu_l = nu_l;
    s->nu_g = nu_g;
}

void or_set_dgdt(or_solver* s, int mode)
{
    s->dgdt = mode;
}

void or_set_chi_case(or_solver* s, int chi_case)
{
    s->chi_case = chi_case;
}

void or_set_body_force(or_solver* s, double gx, double gy)
{
    s->gx = gx;
    s->gy = gy;
}

/* tau_f at a node (reading R8). */
static double tau_f_at(const or_solver* s, long k)
{
    if (s->nu_l > 0 && s->nu_g > 0) {
        double nu = s->phi[k] * (s->nu_l - s->nu_g) + s->nu_g;
        return nu / CS2 + 0.5;
    }
    return s->tau_f;
}

void or_params(const or_solver* s, double out[4])
{
    out[0] = s->beta;
    out[1] = s->kappa;
    out[2] = s->tau_g;
    out[3] = s->alpha;
}

void or_geometry(const or_solver* s, uint8_t* cls, uint8_t* zeta, double* eps,
                 double* av, uint16_t* unknown, uint16_t* doubly)
{
    long N = s->N;
    if (cls) memcpy(cls, s->cls, (size_t)N);
    if (zeta) memcpy(zeta, s->zeta, (size_t)N);
    if (eps) memcpy(eps, s->eps, (size_t)N * sizeof(double));
    if (av) memcpy(av, s->av, (size_t)N * sizeof(double));
    if (unknown || doubly) {
        for (int y = 0; y < s->ny; ++y)
            for (int x = 0; x < s->nx; ++x) {
                long k = (long)y * s->nx + x;
                uint16_t un = 0, db = 0;
                if (s->zeta[k]) {
                    for (int i = 1; i < Q; ++i) {
                        long src = nb(s, x, y, -CX[i], -CY[i]);
                        long dst = nb(s, x, y, CX[i], CY[i]);
                        int src_known = (src >= 0 && s->zeta[src]);
                        int dst_known = (dst >= 0 && s->zeta[dst]);
                        if (!src_known) {
                            un |= (uint16_t)(1u << i);
                            if (!dst_known) db |= (uint16_t)(1u << i);
                        }
                    }
                }
                if (unknown) unknown[k] = un;
                if (doubly) doubly[k] = db;
            }
    }
}

/* ------------------------------------------------------------------------ */
/* Macroscopic fields of the current (post-streaming) state                  */
/* ------------------------------------------------------------------------ */

/* Eq. order-parameter on zeta = 1 nodes. */
static void order_parameter(or_solver* s)
{
    for (long k = 0; k < s->N; ++k) {
        if (!s->zeta[k]) continue;
        double sum = 0.0;
        for (int i = 0; i < Q; ++i) sum += s->g[(long)i * s->N + k];
        s->phi[k] = sum;
    }
}

/* Sec. 2.2.2: phi on ghost nodes from the zeta-weighted mean of the 3x3
 * neighbourhood (b = 9, c'_i = c_i, zeta of the ghost node itself is 0). */
static void ghost_fill(or_solver* s)
{
    for (int y = 0; y < s->ny; ++y)
        for (int x = 0; x < s->nx; ++x) {
            long k = (long)y * s->nx + x;
            if (s->cls[k] == OR_INTERIOR) {
                s->phi[k] = 0.0;
                continue;
            }
            if (s->cls[k] != OR_GHOST) continue;
            if (s->chi_case == 1 || s->chi_case == 3) {
                /* reading R9: Robin condition n_w . grad(phi) = chi on a flat wall */
                long up = nb(s, x, y, 0, 1), dn = nb(s, x, y, 0, -1);
                int zu = (up >= 0 && s->zeta[up]), zd = (dn >= 0 && s->zeta[dn]);
                if (zu != zd) {
                    long b = zu ? up : dn;
                    double c = (s->chi_case == 1 ? -1.0 : 1.0) * sqrt(2.0 * s->beta / s->kappa) * s->costh[b];
                    double pb = s->phi[b];
                    /* d = phi_b - phi_g solves d = c (phi_w - phi_w^2), phi_w = phi_b - d/2 */
                    double A = c / 4.0, B = 1.0 - c * (pb - 0.5), C = c * (pb - pb * pb);
                    double d = 2.0 * C / (B + sqrt(B * B + 4.0 * A * C));
                    s->phi[k] = pb - d;
                    continue;
                }
            }
            double num = 0.0, den = 0.0;
            for (int i = 0; i < Q; ++i) {
                long m = nb(s, x, y, CX[i], CY[i]);
                if (m < 0) continue;
                num += s->zeta[m] * s->phi[m];
                den += s->zeta[m];
            }
            s->phi[k] = num / den;
        }
}

/* Eq. chemical_potencial2 on zeta = 1 nodes:
 * mu = 4 beta phi (phi - 1)(phi - 1/2) - kappa lap(phi)
 *      - a_v sqrt(2 kappa beta) cos(theta) (phi - phi^2). */
static void chemical_potential(or_solver* s)
{
    double root = sqrt(2.0 * s->kappa * s->beta);
    for (int y = 0; y < s->ny; ++y)
        for (int x = 0; x < s->nx; ++x) {
            long k = (long)y * s->nx + x;
            if (!s->zeta[k]) continue;
            double v[3][3];
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    long m = nb(s, x, y, dx, dy);
                    v[dy + 1][dx + 1] = s->phi[m];
                }
            or_stencil(v, &s->gpx[k], &s->gpy[k], &s->lap[k]);
            double ph = s->phi[k];
            /* Table 2: the wall term appears 0, 1 or 2 times (cases 1, 2, 3) */
            double factor = (s->chi_case == 1) ? 0.0 : (s->chi_case == 3 ? 2.0 : 1.0);
            s->mu[k] = 4.0 * s->beta * ph * (ph - 1.0) * (ph - 0.5) - s->kappa * s->lap[k] -
                       factor * s->av[k] * root * s->costh[k] * (ph - ph * ph);
        }
}

/* rho (Sec. 2.1.1), F = F_s = mu grad(phi), u and p (Sec. 2.1.2). */
static void hydro_moments(or_solver* s)
{
    double drho = s->rho_l - s->rho_g;
    for (long k = 0; k < s->N; ++k) {
        if (!s->zeta[k]) continue;
        double fk[Q];
        for (int i = 0; i < Q; ++i) fk[i] = s->f[(long)i * s->N + k];
        double rho = s->phi[k] * drho + s->rho_g;
        double drx = drho * s->gpx[k], dry = drho * s->gpy[k];
        /* F = F_s + F_b, F_s = mu grad(phi), F_b = rho g */
        double Fx = s->mu[k] * s->gpx[k] + rho * s->gx, Fy = s->mu[k] * s->gpy[k] + rho * s->gy;
        or_velocity_pressure(fk, rho, drx, dry, Fx, Fy, &s->ux[k], &s->uy[k], &s->p[k]);
    }
}

static void macroscopic(or_solver* s)
{
    order_parameter(s);
    ghost_fill(s);
    chemical_potential(s);
    hydro_moments(s);
}

/* ------------------------------------------------------------------------ */
/* Initialisation                                                            */
/* ------------------------------------------------------------------------ */

/* Reading R7 plus the first-step history of reading R4. */
static void init_populations(or_solver* s)
{
    ghost_fill(s);
    chemical_potential(s);
    long N = s->N;
    for (long k = 0; k < N; ++k) {
        for (int i = 0; i < Q; ++i) {
            s->f[(long)i * N + k] = 0.0;
            s->g[(long)i * N + k] = 0.0;
        }
        s->s_prev[k] = 0.0;
        if (!s->zeta[k]) continue;
        double geq[Q];
        or_geq(s->phi[k], s->mu[k], s->alpha, geq);
        for (int i = 0; i < Q; ++i) s->g[(long)i * N + k] = geq[i];
    }
    s->history = 0;
    memset(s->budget, 0, sizeof(s->budget));
}

static double periodic_delta(double d, int n, int wrap)
{
    if (!wrap) return d;
    double h = 0.5 * n;
    while (d > h) d -= n;
    while (d < -h) d += n;
    return d;
}

/* Eq. initialphi. */
void or_init_droplet(or_solver* s, double x0, double y0, double R)
{
    for (int y = 0; y < s->ny; ++y)
        for (int x = 0; x < s->nx; ++x) {
            long k = (long)y * s->nx + x;
            if (!s->zeta[k]) {
                if (s->replace_phi) s->phi[k] = 0.0;
                continue;
            }
            double dx = periodic_delta(x - x0, s->nx, 1);
            double dy = periodic_delta(y - y0, s->ny, s->wrap_y);
            double r = sqrt(dx * dx + dy * dy);
            double v = 0.5 + 0.5 * tanh(2.0 * (R - r) / s->W);
            if (s->replace_phi || v > s->phi[k]) s->phi[k] = v;
        }
    s->replace_phi = 0;
    init_populations(s);
}

double or_droplet_phi(double x, double y, double x0, double y0, double R, double W, int nx_period)
{
    double dx = periodic_delta(x - x0, nx_period, nx_period > 0);
    double dy = y - y0;
    double r = sqrt(dx * dx + dy * dy);
    return 0.5 + 0.5 * tanh(2.0 * (R - r) / W);
}

void or_droplet_phi_points(const double* x, const double* y, long n, double x0, double y0,
                           double R, double W, int nx_period, int combine, double* out)
{
    for (long k = 0; k < n; ++k) {
        double v = or_droplet_phi(x[k], y[k], x0, y0, R, W, nx_period);
        if (!combine || v > out[k]) out[k] = v;
    }
}

void or_init_phi(or_solver* s, const double* phi)
{
    for (long k = 0; k < s->N; ++k) s->phi[k] = s->zeta[k] ? phi[k] : 0.0;
    s->replace_phi = 0;
    init_populations(s);
}

/* ------------------------------------------------------------------------ */
/* One time step                                                             */
/* ------------------------------------------------------------------------ */
static void one_step(or_solver* s)
{
    long N = s->N;
    int nx = s->nx, ny = s->ny;
    macroscopic(s);

    double mass_before = 0.0, src_sum = 0.0, lost = 0.0, bb = 0.0;
    for (long k = 0; k < N; ++k)
        if (s->zeta[k]) mass_before += s->phi[k];

    /* Collision of f (Eq. BGK-NS) and g (Eq. BGK) on zeta = 1 nodes. */
    double drho = s->rho_l - s->rho_g;
    for (long k = 0; k < N; ++k) {
        if (!s->zeta[k]) continue;
        double ph = s->phi[k], mu = s->mu[k];
        double ux = s->ux[k], uy = s->uy[k];
        double rho = ph * drho + s->rho_g;
        double drx = drho * s->gpx[k], dry = drho * s->gpy[k];
        double Fx = mu * s->gpx[k] + rho * s->gx, Fy = mu * s->gpy[k] + rho * s->gy;
        double tau = tau_f_at(s, k);

        double feq[Q], Fi[Q];
        or_feq(s->p[k], rho, ux, uy, feq);
        or_force(tau, ux, uy, drx, dry, Fx, Fy, Fi);
        for (int i = 0; i < Q; ++i) {
            double fi = s->f[(long)i * N + k];
            s->fpost[(long)i * N + k] = fi - (fi - feq[i]) / tau + Fi[i];
        }

        double s_now = ux * s->gpx[k] + uy * s->gpy[k];
        double s_old = s->history ? s->s_prev[k] : s_now;
        double geq[Q], G_now[Q], G_old[Q];
        or_geq(ph, mu, s->alpha, geq);
        or_source(s_now, G_now);
        or_source(s_old, G_old);
        for (int i = 0; i < Q; ++i) {
            double gi = s->g[(long)i * N + k];
            double src = (s->dgdt == 1) ? G_now[i] : G_now[i] + 0.5 * (G_now[i] - G_old[i]);
            s->gpost[(long)i * N + k] = gi - (gi - geq[i]) / s->tau_g + src;
            src_sum += src;
        }
        s->s_prev[k] = s_now;
    }

    /* Streaming: f_i(x + c_i, t + 1) = f*_i(x, t); populations that land on
     * zeta = 0 nodes (or leave the domain) are not kept. */
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            long k = (long)y * nx + x;
            if (!s->zeta[k]) continue;
            for (int i = 0; i < Q; ++i) {
                long m = nb(s, x, y, CX[i], CY[i]);
                if (m >= 0 && s->zeta[m]) {
                    s->f[(long)i * N + m] = s->fpost[(long)i * N + k];
                    s->g[(long)i * N + m] = s->gpost[(long)i * N + k];
                } else {
                    lost += s->gpost[(long)i * N + k];
                }
            }
        }

    /* Modified bounce-back (Sec. 2.2.2, reading R6). The known populations
     * were all written above, so the order of this loop does not matter. */
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            long k = (long)y * nx + x;
            if (!s->zeta[k]) continue;
            for (int i = 1; i < Q; ++i) {
                long src = nb(s, x, y, -CX[i], -CY[i]);
                if (src >= 0 && s->zeta[src]) continue; /* known */
                int io = OPP[i];
                long dst = nb(s, x, y, CX[i], CY[i]);
                int opp_known = (dst >= 0 && s->zeta[dst]);
                double fv = opp_known ? s->f[(long)io * N + k] : s->fpost[(long)io * N + k];
                double gv = opp_known ? s->g[(long)io * N + k] : s->gpost[(long)io * N + k];
                s->f[(long)i * N + k] = fv;
                s->g[(long)i * N + k] = gv;
                bb += gv;
            }
        }

    s->budget[0] = mass_before;
    s->budget[1] = src_sum;
    s->budget[2] = lost;
    s->budget[3] = bb;
    s->history = 1;
    s->replace_phi = 1;
    s->steps += 1;
}

void or_step(or_solver* s, long n)
{
    for (long t = 0; t < n; ++t) one_step(s);
}

void or_get(or_solver* s, double* phi, double* u, double* p)
{
    macroscopic(s);
    for (long k = 0; k < s->N; ++k) {
        int z = s->zeta[k];
        if (phi) phi[k] = s->phi[k];
        if (u) {
            u[2 * k] = z ? s->ux[k] : 0.0;
            u[2 * k + 1] = z ? s->uy[k] : 0.0;
        }
        if (p) p[k] = z ? s->p[k] : 0.0;
    }
}

double or_mass(const or_solver* s)
{
    double m = 0.0;
    for (long k = 0; k < s->N; ++k) {
        if (!s->zeta[k]) continue;
        for (int i = 0; i < Q; ++i) m += s->g[(long)i * s->N + k];
    }
    return m;
}

void or_budget(const or_solver* s, double out[4])
{
    for (int i = 0; i < 4; ++i) out[i] = s->budget[i];
}

void or_state(const or_solver* s, double* f, double* g, double* s_prev)
{
    size_t n = (size_t)(Q * s->N) * sizeof(double);
    if (f) memcpy(f, s->f, n);
    if (g) memcpy(g, s->g, n);
    if (s_prev) memcpy(s_prev, s->s_prev, (size_t)s->N * sizeof(double));
}

void or_set_state(or_solver* s, const double* f, const double* g)
{
    size_t n = (size_t)(Q * s->N) * sizeof(double);
    memcpy(s->f, f, n);
    memcpy(s->g, g, n);
}

long or_steps(const or_solver* s)
{
    return s->steps;
}

/* ------------------------------------------------------------------------ */
/* Contact angle (a reading: the paper does not state its measurement)       */
/* ------------------------------------------------------------------------ */

/* Solve the 3x3 system A z = b by Gaussian elimination with partial pivoting. */
static int solve3(double A[3][3], double b[3], double z[3])
{
    for (int c = 0; c < 3; ++c) {
        int piv = c;
        for (int r = c + 1; r < 3; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (A[piv][c] == 0.0) return -1;
        if (piv != c) {
            for (int k = 0; k < 3; ++k) {
                double t = A[c][k];
                A[c][k] = A[piv][k];
                A[piv][k] = t;
            }
            double t = b[c];
            b[c] = b[piv];
            b[piv] = t;
        }
        for (int r = c + 1; r < 3; ++r) {
            double m = A[r][c] / A[c][c];
            for (int k = c; k < 3; ++k) A[r][k] -= m * A[c][k];
            b[r] -= m * b[c];
        }
    }
    for (int r = 2; r >= 0; --r) {
        double acc = b[r];
        for (int k = r + 1; k < 3; ++k) acc -= A[r][k] * z[k];
        z[r] = acc / A[r][r];
    }
    return 0;
}

/* Algebraic circle fit (minimise sum (x^2 + y^2 + D x + E y + F)^2) on
 * coordinates taken relative to the point mean, then Gauss-Newton on the
 * geometric residual |q - centre| - R. */
int or_circle_fit(const double* x, const double* y, int n, double circle[3])
{
    if (n < 3) return -1;
    double mx = 0.0, my = 0.0;
    for (int k = 0; k < n; ++k) {
        mx += x[k];
        my += y[k];
    }
    mx /= n;
    my /= n;
    double A[3][3] = {{0}}, b[3] = {0};
    for (int k = 0; k < n; ++k) {
        double u = x[k] - mx, v = y[k] - my;
        double row[3] = {u, v, 1.0};
        double rhs = -(u * u + v * v);
        for (int r = 0; r < 3; ++r) {
            for (int c = 0; c < 3; ++c) A[r][c] += row[r] * row[c];
            b[r] += row[r] * rhs;
        }
    }
    double z[3];
    if (solve3(A, b, z)) return -1;
    double a = -z[0] / 2.0, bb = -z[1] / 2.0;
    double R2 = a * a + bb * bb - z[2];
    if (!(R2 > 0)) return -1;
    double R = sqrt(R2);
    for (int it = 0; it < 50; ++it) {
        double JJ[3][3] = {{0}}, Jr[3] = {0};
        for (int k = 0; k < n; ++k) {
            double u = x[k] - mx - a, v = y[k] - my - bb;
            double d = sqrt(u * u + v * v);
            if (d == 0.0) continue;
            double J[3] = {-u / d, -v / d, -1.0};
            double r = d - R;
            for (int p = 0; p < 3; ++p) {
                for (int q = 0; q < 3; ++q) JJ[p][q] += J[p] * J[q];
                Jr[p] -= J[p] * r;
            }
        }
        double dz[3];
        if (solve3(JJ, Jr, dz)) break;
        a += dz[0];
        bb += dz[1];
        R += dz[2];
        if (fabs(dz[0]) + fabs(dz[1]) + fabs(dz[2]) < 1e-13 * (1.0 + fabs(R))) break;
    }
    circle[0] = a + mx;
    circle[1] = bb + my;
    circle[2] = R;
    return 0;
}

static double wall_distance(const or_wall* w, double x, double y)
{
    if (w->type == 0) return (x - w->px) * w->nx_ + (y - w->py) * w->ny_;
    double dx = x - w->px, dy = y - w->py;
    return sqrt(dx * dx + dy * dy) - w->r;
}

int or_contact_angle(const double* phi, const uint8_t* cls, int nx, int ny,
                     const or_wall* wall, double* theta_deg, double circle[3])
{
    long cap = 2L * nx * ny;
    double* px = (double*)xcalloc(cap, sizeof(double));
    double* py = (double*)xcalloc(cap, sizeof(double));
    int n = 0;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            long k = (long)y * nx + x;
            if (cls[k] != OR_FLUID) continue;
            double a = phi[k];
            /* right neighbour (no wrap) and upper neighbour */
            for (int dir = 0; dir < 2; ++dir) {
                int xx = x + (dir == 0), yy = y + (dir == 1);
                if (xx >= nx || yy >= ny) continue;
                long m = (long)yy * nx + xx;
                if (cls[m] != OR_FLUID) continue;
                double b = phi[m];
                if ((a >= 0.5) == (b >= 0.5)) continue;
                double t = (0.5 - a) / (b - a);
                double qx = x + (dir == 0 ? t : 0.0);
                double qy = y + (dir == 1 ? t : 0.0);
                if (qx < wall->x_lo || qx >= wall->x_hi) continue;
                if (wall_distance(wall, qx, qy) <= wall->exclude) continue;
                px[n] = qx;
                py[n] = qy;
                ++n;
            }
        }
    int used = n;
    if (n < 3 || or_circle_fit(px, py, n, circle)) {
        used = (n < 3) ? n : 0;
        free(px);
        free(py);
        *theta_deg = NAN;
        return used;
    }
    double ct;
    if (wall->type == 0) {
        double dc = (circle[0] - wall->px) * wall->nx_ + (circle[1] - wall->py) * wall->ny_;
        ct = -dc / circle[2];
    } else {
        double dx = circle[0] - wall->px, dy = circle[1] - wall->py;
        double D2 = dx * dx + dy * dy;
        ct = (circle[2] * circle[2] + wall->r * wall->r - D2) / (2.0 * circle[2] * wall->r);
    }
    if (ct > 1.0) ct = 1.0;
    if (ct < -1.0) ct = -1.0;
    *theta_deg = acos(ct) * 180.0 / M_PI;
    free(px);
    free(py);
    return used;
}
