/*
 * pflbm_oracle3d.c -- plain FP64 CPU oracle of the 3D scheme (see
 * pflbm_oracle3d.h). TEST INFRASTRUCTURE. Same algorithm and readings as the
 * 2D oracle (pflbm_oracle.c, readings R1-R7), with these 3D specifics:
 *   - f on D3Q19 (Eq. 3ci, w = 1/3, 1/18, 1/36, c_s^2 = 1/3); g on D3Q7
 *     (w = 1/4, 1/8, c_s^2 = 1/4), so alpha = M / (c_s^2 (tau_g - 1/2)) uses
 *     1/4 and the source of Eq. F_i uses I:(c c - c_s^2 I) = |c|^2 - 3 c_s^2;
 *   - gradients and Laplacians (Eqs. gradient, Laplace), and a_v = |grad
 *     epsilon|, use the D3Q19 weights;
 *   - R3D: a solid node with a non-solid D3Q19 neighbour is a boundary node
 *     (zeta = 1); another solid node with a zeta = 1 D3Q19 neighbour is a
 *     ghost, whose phi is the zeta-weighted mean of its 27-neighbourhood
 *     (Sec. 2.2.2, b = 27); the rest are interior nodes.
 */
#include "pflbm_oracle3d.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define Q19 19
#define Q7 7
static const double CS2F = 1.0 / 3.0; /* D3Q19 */
static const double CS2G = 1.0 / 4.0; /* D3Q7 */

static const int C19[Q19][3] = {
    {0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1},
    {-1, 0, 1}, {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
static const int C7[Q7][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};

static double W19(int i) { return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }
static double W7(int i) { return i == 0 ? 1.0 / 4.0 : 1.0 / 8.0; }

static int opp19(int i)
{
    for (int j = 0; j < Q19; ++j)
        if (C19[j][0] == -C19[i][0] && C19[j][1] == -C19[i][1] && C19[j][2] == -C19[i][2]) return j;
    return -1;
}
static int opp7(int i)
{
    for (int j = 0; j < Q7; ++j)
        if (C7[j][0] == -C7[i][0] && C7[j][1] == -C7[i][1] && C7[j][2] == -C7[i][2]) return j;
    return -1;
}

void or3_lattices(int c19[19][3], double w19[19], int c7[7][3], double w7[7])
{
    for (int i = 0; i < Q19; ++i) {
        for (int d = 0; d < 3; ++d) c19[i][d] = C19[i][d];
        w19[i] = W19(i);
    }
    for (int i = 0; i < Q7; ++i) {
        for (int d = 0; d < 3; ++d) c7[i][d] = C7[i][d];
        w7[i] = W7(i);
    }
}

static double dot3(const int c[3], const double v[3]) { return c[0] * v[0] + c[1] * v[1] + c[2] * v[2]; }

/* s_i(u), Eq. Siu, on D3Q19 */
static double s_i3(int i, const double u[3])
{
    double cu = dot3(C19[i], u);
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return W19(i) * (cu / CS2F + cu * cu / (2.0 * CS2F * CS2F) - uu / (2.0 * CS2F));
}

/* Eq. feq_i */
void or3_feq(double p, double rho, const double u[3], double feq[19])
{
    for (int i = 0; i < Q19; ++i)
        feq[i] = (i == 0 ? p / CS2F * (W19(0) - 1.0) : p / CS2F * W19(i)) + rho * s_i3(i, u);
}

/* Eq. H_i on D3Q7 */
void or3_geq(double phi, double mu, double alpha, double geq[7])
{
    geq[0] = phi - (1.0 - W7(0)) * alpha * mu;
    for (int i = 1; i < Q7; ++i) geq[i] = W7(i) * alpha * mu;
}

/* Eq. GGi (prefactor with tau_f) on D3Q19 */
void or3_force(double tau_f, const double u[3], const double drho[3], const double F[3], double Fi[19])
{
    double pre = 1.0 - 1.0 / (2.0 * tau_f);
    double ugr = u[0] * drho[0] + u[1] * drho[1] + u[2] * drho[2];
    for (int i = 0; i < Q19; ++i) {
        double cF = dot3(C19[i], F), cu = dot3(C19[i], u), cdr = dot3(C19[i], drho);
        Fi[i] = pre * W19(i) * (ugr + cF / CS2F + (cu * cdr - CS2F * ugr) / CS2F);
    }
}

/* Eq. F_i on D3Q7: I:(c c - c_s^2 I) = |c|^2 - 3 c_s^2 */
void or3_source(double s, double Gi[7])
{
    for (int i = 0; i < Q7; ++i) {
        double c2 = (double)(C7[i][0] * C7[i][0] + C7[i][1] * C7[i][1] + C7[i][2] * C7[i][2]);
        Gi[i] = W7(i) * s * (-1.0 + (c2 - 3.0 * CS2G) / (2.0 * CS2G));
    }
}

void or3_velocity_pressure(const double f[19], double rho, const double drho[3], const double F[3],
                           double u[3], double* p)
{
    double m[3] = {0, 0, 0};
    for (int i = 0; i < Q19; ++i)
        for (int d = 0; d < 3; ++d) m[d] += C19[i][d] * f[i];
    for (int d = 0; d < 3; ++d) u[d] = (m[d] + 0.5 * F[d]) / rho;
    double sum = 0.0;
    for (int i = 1; i < Q19; ++i) sum += f[i];
    *p = CS2F / (1.0 - W19(0)) * (sum + 0.5 * (u[0] * drho[0] + u[1] * drho[1] + u[2] * drho[2]) + rho * s_i3(0, u));
}

void or3_stencil(const double v[3][3][3], double g[3], double* lap)
{
    double v0 = v[1][1][1];
    g[0] = g[1] = g[2] = 0.0;
    double l = 0.0;
    for (int i = 1; i < Q19; ++i) {
        double vi = v[C19[i][2] + 1][C19[i][1] + 1][C19[i][0] + 1];
        for (int d = 0; d < 3; ++d) g[d] += W19(i) * C19[i][d] * vi / CS2F;
        l += 2.0 * W19(i) * (vi - v0) / CS2F;
    }
    *lap = l;
}

/* ------------------------------------------------------------------------ */
enum { F3 = 0, B3 = 1, G3 = 2, I3 = 3 };

struct or3_solver {
    int nx, ny, nz, wrap_z;
    long N;
    double sigma, W, M, tau_f, tau_g, rho_l, rho_g, beta, kappa, alpha, costh;
    uint8_t *cls, *zeta;
    double *eps, *av;
    double *f, *g, *fpost, *gpost, *s_prev;
    double *phi, *mu, *gp, *ux, *p;   /* gp: [N][3], ux: [N][3] */
    int history, replace_phi;
    int dgdt;                         /* 1: the (1/2) dG/dt term omitted */
    double budget[4];
};

static long nb3(const or3_solver* s, int x, int y, int z, int dx, int dy, int dz)
{
    int xx = (x + dx) % s->nx, yy = (y + dy) % s->ny, zz = z + dz;
    if (xx < 0) xx += s->nx;
    if (yy < 0) yy += s->ny;
    if (s->wrap_z) {
        zz %= s->nz;
        if (zz < 0) zz += s->nz;
    } else if (zz < 0 || zz >= s->nz) {
        return -1;
    }
    return ((long)zz * s->ny + yy) * s->nx + xx;
}

#define FOR_NODES(s)                          \
    for (int z = 0; z < (s)->nz; ++z)         \
        for (int y = 0; y < (s)->ny; ++y)     \
            for (int x = 0; x < (s)->nx; ++x)

#define KIDX(s) (((long)z * (s)->ny + y) * (s)->nx + x)

static void classify3(or3_solver* s, const uint8_t* solid)
{
    FOR_NODES(s)
    {
        long k = KIDX(s);
        if (!solid[k]) {
            s->cls[k] = F3;
            continue;
        }
        int touches = 0;
        for (int i = 1; i < Q19; ++i) {
            long m = nb3(s, x, y, z, C19[i][0], C19[i][1], C19[i][2]);
            if (m >= 0 && !solid[m]) touches = 1;
        }
        s->cls[k] = touches ? B3 : I3;
    }
    for (long k = 0; k < s->N; ++k) s->zeta[k] = (s->cls[k] == F3 || s->cls[k] == B3);
    FOR_NODES(s)
    {
        long k = KIDX(s);
        if (s->cls[k] != I3) continue;
        for (int i = 1; i < Q19; ++i) {
            long m = nb3(s, x, y, z, C19[i][0], C19[i][1], C19[i][2]);
            if (m >= 0 && s->zeta[m]) s->cls[k] = G3;
        }
    }
    for (long k = 0; k < s->N; ++k) s->eps[k] = s->cls[k] == F3 ? 1.0 : 0.0;
    FOR_NODES(s)
    {
        long k = KIDX(s);
        s->av[k] = 0.0;
        if (!s->zeta[k]) continue;
        double v[3][3][3];
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    long m = nb3(s, x, y, z, dx, dy, dz);
                    v[dz + 1][dy + 1][dx + 1] = m >= 0 ? s->eps[m] : 0.0;
                }
        double gr[3], lap;
        or3_stencil(v, gr, &lap);
        s->av[k] = sqrt(gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2]);
    }
}

or3_solver* or3_create(int nx, int ny, int nz, int wrap_z, const uint8_t* solid, double theta_deg,
                       double sigma, double W, double M, double tau_f, double rho_l, double rho_g,
                       double tau_g)
{
    if (nx < 3 || ny < 3 || nz < 3 || !solid || !(W > 0) || !(M > 0) || !(tau_f > 0.5) || !(rho_l > 0) ||
        !(rho_g > 0) || !(sigma >= 0))
        return NULL;
    if (tau_g <= 0) tau_g = 1.0;
    long plane = (long)nx * ny;
    if (!wrap_z) {
        for (long k = 0; k < plane; ++k)
            if (!solid[k] || !solid[plane + k] || !solid[(long)(nz - 2) * plane + k] ||
                !solid[(long)(nz - 1) * plane + k])
                return NULL;
    }
    or3_solver* s = (or3_solver*)calloc(1, sizeof(or3_solver));
    s->nx = nx;
    s->ny = ny;
    s->nz = nz;
    s->wrap_z = wrap_z ? 1 : 0;
    s->N = plane * nz;
    s->sigma = sigma;
    s->W = W;
    s->M = M;
    s->tau_f = tau_f;
    s->tau_g = tau_g;
    s->rho_l = rho_l;
    s->rho_g = rho_g;
    s->beta = 12.0 * sigma / W;
    s->kappa = 1.5 * sigma * W;
    s->alpha = M / (CS2G * (tau_g - 0.5));
    s->costh = cos(theta_deg * M_PI / 180.0);
    long N = s->N;
    s->cls = (uint8_t*)calloc(N, 1);
    s->zeta = (uint8_t*)calloc(N, 1);
    s->eps = (double*)calloc(N, sizeof(double));
    s->av = (double*)calloc(N, sizeof(double));
    s->f = (double*)calloc(Q19 * N, sizeof(double));
    s->fpost = (double*)calloc(Q19 * N, sizeof(double));
    s->g = (double*)calloc(Q7 * N, sizeof(double));
    s->gpost = (double*)calloc(Q7 * N, sizeof(double));
    s->s_prev = (double*)calloc(N, sizeof(double));
    s->phi = (double*)calloc(N, sizeof(double));
    s->mu = (double*)calloc(N, sizeof(double));
    s->gp = (double*)calloc(3 * N, sizeof(double));
    s->ux = (double*)calloc(3 * N, sizeof(double));
    s->p = (double*)calloc(N, sizeof(double));
    classify3(s, solid);
    s->replace_phi = 1;
    return s;
}

void or3_destroy(or3_solver* s)
{
    if (!s) return;
    free(s->cls);
    free(s->zeta);
    free(s->eps);
    free(s->av);
    free(s->f);
    free(s->fpost);
    free(s->g);
    free(s->gpost);
    free(s->s_prev);
    free(s->phi);
    free(s->mu);
    free(s->gp);
    free(s->ux);
    free(s->p);
    free(s);
}

void or3_params(const or3_solver* s, double out[4])
{
    out[0] = s->beta;
    out[1] = s->kappa;
    out[2] = s->tau_g;
    out[3] = s->alpha;
}

void or3_geometry(const or3_solver* s, uint8_t* cls, double* av)
{
    if (cls) memcpy(cls, s->cls, (size_t)s->N);
    if (av) memcpy(av, s->av, (size_t)s->N * sizeof(double));
}

/* ---- macroscopic fields ---- */
static void macro3(or3_solver* s)
{
    long N = s->N;
    for (long k = 0; k < N; ++k) {
        if (!s->zeta[k]) continue;
        double sum = 0.0;
        for (int i = 0; i < Q7; ++i) sum += s->g[(long)i * N + k];
        s->phi[k] = sum;
    }
    /* ghost average over the 27-neighbourhood (Sec. 2.2.2, b = 27) */
    FOR_NODES(s)
    {
        long k = KIDX(s);
        if (s->cls[k] == I3) {
            s->phi[k] = 0.0;
            continue;
        }
        if (s->cls[k] != G3) continue;
        double num = 0.0, den = 0.0;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    long m = nb3(s, x, y, z, dx, dy, dz);
                    if (m < 0) continue;
                    num += s->zeta[m] * s->phi[m];
                    den += s->zeta[m];
                }
        s->phi[k] = num / den;
    }
    double root = sqrt(2.0 * s->kappa * s->beta), drho = s->rho_l - s->rho_g;
    FOR_NODES(s)
    {
        long k = KIDX(s);
        if (!s->zeta[k]) continue;
        double v[3][3][3];
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) v[dz + 1][dy + 1][dx + 1] = s->phi[nb3(s, x, y, z, dx, dy, dz)];
        double lap;
        or3_stencil(v, &s->gp[3 * k], &lap);
        double ph = s->phi[k];
        s->mu[k] = 4.0 * s->beta * ph * (ph - 1.0) * (ph - 0.5) - s->kappa * lap -
                   s->av[k] * root * s->costh * (ph - ph * ph);
        double fk[Q19];
        for (int i = 0; i < Q19; ++i) fk[i] = s->f[(long)i * N + k];
        double rho = ph * drho + s->rho_g;
        double dr[3] = {drho * s->gp[3 * k], drho * s->gp[3 * k + 1], drho * s->gp[3 * k + 2]};
        double F[3] = {s->mu[k] * s->gp[3 * k], s->mu[k] * s->gp[3 * k + 1], s->mu[k] * s->gp[3 * k + 2]};
        or3_velocity_pressure(fk, rho, dr, F, &s->ux[3 * k], &s->p[k]);
    }
}

static void init_pop3(or3_solver* s)
{
    /* ghost fill and mu of the initial phi, then f = 0, g = g^eq (reading R7) */
    long N = s->N;
    for (long k = 0; k < N; ++k) {
        s->s_prev[k] = 0.0;
        for (int i = 0; i < Q19; ++i) s->f[(long)i * N + k] = 0.0;
    }
    /* the macroscopic pass recomputes phi from g: set g so that sum g = phi first */
    for (long k = 0; k < N; ++k) {
        for (int i = 0; i < Q7; ++i) s->g[(long)i * N + k] = 0.0;
        if (s->zeta[k]) s->g[k] = s->phi[k];
    }
    macro3(s);
    for (long k = 0; k < N; ++k) {
        if (!s->zeta[k]) continue;
        double geq[Q7];
        or3_geq(s->phi[k], s->mu[k], s->alpha, geq);
        for (int i = 0; i < Q7; ++i) s->g[(long)i * N + k] = geq[i];
    }
    s->history = 0;
}

void or3_init_droplet(or3_solver* s, double x0, double y0, double z0, double R)
{
    FOR_NODES(s)
    {
        long k = KIDX(s);
        if (!s->zeta[k]) {
            if (s->replace_phi) s->phi[k] = 0.0;
            continue;
        }
        double dx = x - x0, dy = y - y0;
        while (dx > 0.5 * s->nx) dx -= s->nx;
        while (dx < -0.5 * s->nx) dx += s->nx;
        while (dy > 0.5 * s->ny) dy -= s->ny;
        while (dy < -0.5 * s->ny) dy += s->ny;
        double dz = z - z0;
        if (s->wrap_z) {
            while (dz > 0.5 * s->nz) dz -= s->nz;
            while (dz < -0.5 * s->nz) dz += s->nz;
        }
        double r = sqrt(dx * dx + dy * dy + dz * dz);
        double v = 0.5 + 0.5 * tanh(2.0 * (R - r) / s->W);
        if (s->replace_phi || v > s->phi[k]) s->phi[k] = v;
    }
    s->replace_phi = 0;
    init_pop3(s);
}

void or3_init_phi(or3_solver* s, const double* phi)
{
    for (long k = 0; k < s->N; ++k) s->phi[k] = s->zeta[k] ? phi[k] : 0.0;
    s->replace_phi = 0;
    init_pop3(s);
}

static void step3(or3_solver* s)
{
    long N = s->N;
    macro3(s);
    double mass = 0.0, src_sum = 0.0, lost = 0.0, bb = 0.0;
    for (long k = 0; k < N; ++k)
        if (s->zeta[k]) mass += s->phi[k];
    double drho = s->rho_l - s->rho_g;
    for (long k = 0; k < N; ++k) {
        if (!s->zeta[k]) continue;
        double ph = s->phi[k], mu = s->mu[k], *u = &s->ux[3 * k], *gp = &s->gp[3 * k];
        double rho = ph * drho + s->rho_g;
        double dr[3] = {drho * gp[0], drho * gp[1], drho * gp[2]};
        double F[3] = {mu * gp[0], mu * gp[1], mu * gp[2]};
        double feq[Q19], Fi[Q19];
        or3_feq(s->p[k], rho, u, feq);
        or3_force(s->tau_f, u, dr, F, Fi);
        for (int i = 0; i < Q19; ++i) {
            double fi = s->f[(long)i * N + k];
            s->fpost[(long)i * N + k] = fi - (fi - feq[i]) / s->tau_f + Fi[i];
        }
        double s_now = u[0] * gp[0] + u[1] * gp[1] + u[2] * gp[2];
        double s_old = (s->history && !s->dgdt) ? s->s_prev[k] : s_now;
        double geq[Q7], Gn[Q7], Go[Q7];
        or3_geq(ph, mu, s->alpha, geq);
        or3_source(s_now, Gn);
        or3_source(s_old, Go);
        for (int i = 0; i < Q7; ++i) {
            double gi = s->g[(long)i * N + k];
            double src = Gn[i] + 0.5 * (Gn[i] - Go[i]);
            s->gpost[(long)i * N + k] = gi - (gi - geq[i]) / s->tau_g + src;
            src_sum += src;
        }
        s->s_prev[k] = s_now;
    }
    /* streaming */
    FOR_NODES(s)
    {
        long k = KIDX(s);
        if (!s->zeta[k]) continue;
        for (int i = 0; i < Q19; ++i) {
            long m = nb3(s, x, y, z, C19[i][0], C19[i][1], C19[i][2]);
            if (m >= 0 && s->zeta[m]) s->f[(long)i * N + m] = s->fpost[(long)i * N + k];
        }
        for (int i = 0; i < Q7; ++i) {
            long m = nb3(s, x, y, z, C7[i][0], C7[i][1], C7[i][2]);
            if (m >= 0 && s->zeta[m])
                s->g[(long)i * N + m] = s->gpost[(long)i * N + k];
            else
                lost += s->gpost[(long)i * N + k];
        }
    }
    /* modified bounce-back (R6) on each lattice */
    FOR_NODES(s)
    {
        long k = KIDX(s);
        if (!s->zeta[k]) continue;
        for (int i = 1; i < Q19; ++i) {
            long src = nb3(s, x, y, z, -C19[i][0], -C19[i][1], -C19[i][2]);
            if (src >= 0 && s->zeta[src]) continue;
            int io = opp19(i);
            long dst = nb3(s, x, y, z, C19[i][0], C19[i][1], C19[i][2]);
            int ok = dst >= 0 && s->zeta[dst];
            s->f[(long)i * N + k] = ok ? s->f[(long)io * N + k] : s->fpost[(long)io * N + k];
        }
        for (int i = 1; i < Q7; ++i) {
            long src = nb3(s, x, y, z, -C7[i][0], -C7[i][1], -C7[i][2]);
            if (src >= 0 && s->zeta[src]) continue;
            int io = opp7(i);
            long dst = nb3(s, x, y, z, C7[i][0], C7[i][1], C7[i][2]);
            int ok = dst >= 0 && s->zeta[dst];
            double v = ok ? s->g[(long)io * N + k] : s->gpost[(long)io * N + k];
            s->g[(long)i * N + k] = v;
            bb += v;
        }
    }
    s->budget[0] = mass;
    s->budget[1] = src_sum;
    s->budget[2] = lost;
    s->budget[3] = bb;
    s->history = 1;
    s->replace_phi = 1;
}

void or3_set_dgdt(or3_solver* s, int mode) { s->dgdt = mode ? 1 : 0; }

void or3_step(or3_solver* s, long n)
{
    for (long t = 0; t < n; ++t) step3(s);
}

void or3_get(or3_solver* s, double* phi, double* u, double* p)
{
    macro3(s);
    for (long k = 0; k < s->N; ++k) {
        int z = s->zeta[k];
        if (phi) phi[k] = s->phi[k];
        if (u)
            for (int d = 0; d < 3; ++d) u[3 * k + d] = z ? s->ux[3 * k + d] : 0.0;
        if (p) p[k] = z ? s->p[k] : 0.0;
    }
}

double or3_mass(const or3_solver* s)
{
    double m = 0.0;
    for (long k = 0; k < s->N; ++k) {
        if (!s->zeta[k]) continue;
        for (int i = 0; i < Q7; ++i) m += s->g[(long)i * s->N + k];
    }
    return m;
}

void or3_budget(const or3_solver* s, double out[4])
{
    for (int i = 0; i < 4; ++i) out[i] = s->budget[i];
}

/* ---- sphere fit for a cap on a flat wall ---- */
static int solve4(double A[4][4], double b[4], double x[4])
{
    for (int c = 0; c < 4; ++c) {
        int piv = c;
        for (int r = c + 1; r < 4; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (A[piv][c] == 0.0) return -1;
        for (int k = 0; k < 4; ++k) {
            double t = A[c][k];
            A[c][k] = A[piv][k];
            A[piv][k] = t;
        }
        double t = b[c];
        b[c] = b[piv];
        b[piv] = t;
        for (int r = c + 1; r < 4; ++r) {
            double m = A[r][c] / A[c][c];
            for (int k = c; k < 4; ++k) A[r][k] -= m * A[c][k];
            b[r] -= m * b[c];
        }
    }
    for (int r = 3; r >= 0; --r) {
        double acc = b[r];
        for (int k = r + 1; k < 4; ++k) acc -= A[r][k] * x[k];
        x[r] = acc / A[r][r];
    }
    return 0;
}

static double wall_distance3(const or3_wall_t* w, const double q[3])
{
    if (w->type == 0)
        return (q[0] - w->p[0]) * w->n[0] + (q[1] - w->p[1]) * w->n[1] + (q[2] - w->p[2]) * w->n[2];
    double d[3] = {q[0] - w->p[0], q[1] - w->p[1], q[2] - w->p[2]};
    return sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) - w->r;
}

int or3_contact_angle(const double* phi, const uint8_t* cls, int nx, int ny, int nz, const or3_wall_t* wall,
                      double* theta_deg, double sphere[4])
{
    long N = (long)nx * ny * nz, cap = 3 * N;
    double* P = (double*)calloc((size_t)(3 * cap), sizeof(double));
    int n = 0;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long k = ((long)z * ny + y) * nx + x;
                if (cls[k] != F3) continue;
                for (int d = 0; d < 3; ++d) {
                    int xx = x + (d == 0), yy = y + (d == 1), zz = z + (d == 2);
                    if (xx >= nx || yy >= ny || zz >= nz) continue;
                    long m = ((long)zz * ny + yy) * nx + xx;
                    if (cls[m] != F3) continue;
                    double a = phi[k], b = phi[m];
                    if ((a >= 0.5) == (b >= 0.5)) continue;
                    double t = (0.5 - a) / (b - a);
                    double q[3] = {x + (d == 0 ? t : 0.0), y + (d == 1 ? t : 0.0), z + (d == 2 ? t : 0.0)};
                    if (q[0] < wall->x_lo || q[0] >= wall->x_hi || q[1] < wall->y_lo || q[1] >= wall->y_hi) continue;
                    if (wall_distance3(wall, q) <= wall->exclude) continue;
                    P[3 * n] = q[0];
                    P[3 * n + 1] = q[1];
                    P[3 * n + 2] = q[2];
                    ++n;
                }
            }
    if (n < 4) {
        free(P);
        *theta_deg = NAN;
        return n;
    }
    double mc[3] = {0, 0, 0};
    for (int k = 0; k < n; ++k)
        for (int d = 0; d < 3; ++d) mc[d] += P[3 * k + d] / n;
    /* algebraic fit: |q|^2 + D.q + F = 0 on centred points */
    double A[4][4] = {{0}}, b[4] = {0}, z4[4];
    for (int k = 0; k < n; ++k) {
        double r[4] = {P[3 * k] - mc[0], P[3 * k + 1] - mc[1], P[3 * k + 2] - mc[2], 1.0};
        double rhs = -(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        for (int i = 0; i < 4; ++i) {
            for (int j = 0; j < 4; ++j) A[i][j] += r[i] * r[j];
            b[i] += r[i] * rhs;
        }
    }
    if (solve4(A, b, z4)) {
        free(P);
        *theta_deg = NAN;
        return 0;
    }
    double c[3] = {-z4[0] / 2, -z4[1] / 2, -z4[2] / 2};
    double R = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2] - z4[3]);
    for (int it = 0; it < 50; ++it) {
        double JJ[4][4] = {{0}}, Jr[4] = {0}, dz[4];
        for (int k = 0; k < n; ++k) {
            double u[3] = {P[3 * k] - mc[0] - c[0], P[3 * k + 1] - mc[1] - c[1], P[3 * k + 2] - mc[2] - c[2]};
            double dd = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
            if (dd == 0) continue;
            double J[4] = {-u[0] / dd, -u[1] / dd, -u[2] / dd, -1.0}, r = dd - R;
            for (int i = 0; i < 4; ++i) {
                for (int j = 0; j < 4; ++j) JJ[i][j] += J[i] * J[j];
                Jr[i] -= J[i] * r;
            }
        }
        if (solve4(JJ, Jr, dz)) break;
        for (int d = 0; d < 3; ++d) c[d] += dz[d];
        R += dz[3];
        if (fabs(dz[0]) + fabs(dz[1]) + fabs(dz[2]) + fabs(dz[3]) < 1e-13 * (1 + R)) break;
    }
    for (int d = 0; d < 3; ++d) sphere[d] = c[d] + mc[d];
    sphere[3] = R;
    double ct;
    if (wall->type == 0) {
        ct = -((sphere[0] - wall->p[0]) * wall->n[0] + (sphere[1] - wall->p[1]) * wall->n[1] +
               (sphere[2] - wall->p[2]) * wall->n[2]) / R;
    } else {
        double d[3] = {sphere[0] - wall->p[0], sphere[1] - wall->p[1], sphere[2] - wall->p[2]};
        ct = (R * R + wall->r * wall->r - (d[0] * d[0] + d[1] * d[1] + d[2] * d[2])) / (2.0 * R * wall->r);
    }
    ct = ct > 1 ? 1 : (ct < -1 ? -1 : ct);
    *theta_deg = acos(ct) * 180.0 / M_PI;
    free(P);
    return n;
}

int or3_contact_angle_flat(const double* phi, const uint8_t* cls, int nx, int ny, int nz, double zw,
                           double exclude, double* theta_deg, double sphere[4])
{
    or3_wall_t w;
    memset(&w, 0, sizeof(w));
    w.type = 0;
    w.p[2] = zw;
    w.n[2] = 1.0;
    w.x_lo = w.y_lo = -1e300;
    w.x_hi = w.y_hi = 1e300;
    w.exclude = exclude;
    return or3_contact_angle(phi, cls, nx, ny, nz, &w, theta_deg, sphere);
}
