/*
 * pflbm.h -- C ABI of the GB300 (sm_103a) phase-field lattice Boltzmann
 * library for droplets on wetting walls, after arXiv 2312.00369 (Ju, Guo,
 * Yan, Sun): a Cahn-Hilliard phase lattice g_i and a pressure-based
 * hydrodynamic lattice f_i on D2Q9, coupled by the surface-tension force
 * mu grad(phi), with the liquid-solid surface energy folded into the chemical
 * potential (Eq. chemical_potencial2) and a zero-normal-gradient ghost average
 * on solid nodes (Sec. 2.2.2).
 *
 * General conventions
 *  - Lattice units: dx = dt = 1, c_s^2 = 1/3. Fields are row-major [ny][nx],
 *    node (x, y) at index y*nx + x. x is periodic; rows 0, 1, ny-2 and ny-1
 *    must be solid (so every node that collides has all 8 neighbours).
 *  - Every call returns a status (PFLBM_OK = 0 or a negative code); no C++
 *    exception crosses the ABI. pflbm_last_error() gives a text for the last
 *    failure of the calling thread.
 *  - Host arrays passed in are copied and never retained; output buffers are
 *    owned by the caller. A handle is not thread-safe: use one handle from one
 *    thread at a time. All device work of a handle runs on its stream.
 *  - Parameters follow the paper's statement of the problem: contact angle
 *    theta (Eq. b1), surface tension sigma and interface width W (Eq.
 *    initialphi), mobility M (Eq. mobility), relaxation time tau_f with
 *    nu = c_s^2 (tau_f - 1/2), densities rho_l (phi = 1) and rho_g (phi = 0)
 *    (Sec. 2.1.1). Derived: beta = 12 sigma / W, kappa = 3 sigma W / 2 (the
 *    unique pair for which the tanh profile of width W is the flat-interface
 *    equilibrium and sigma = sqrt(2 kappa beta)/6), tau_g = 1 unless given,
 *    alpha = M / (c_s^2 (tau_g - 1/2)).
 */
#ifndef PFLBM_H
#define PFLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pflbm pflbm_t; /* opaque, owned by the library */

enum pflbm_status {
    PFLBM_OK = 0,
    PFLBM_EINVAL = -1,   /* invalid argument or handle                       */
    PFLBM_ENOMEM = -2,   /* device allocation failed                         */
    PFLBM_EBADMASK = -3, /* rows 0, 1, ny-2, ny-1 of the mask are not solid  */
    PFLBM_ENUMERIC = -4, /* NaN or |u| >= 0.3 seen on the device             */
    PFLBM_ETIMEOUT = -5, /* a bounded wait of the staged step kernel for its
                            TMA data gave up (the kernel then returns)       */
    PFLBM_ECUDA = -6     /* a CUDA runtime call failed                       */
};

/* Storage precision of the populations. Collision and stencils run in FP64
 * for PFLBM_FP64 and in FP32 otherwise; the 16-bit modes store f_i and
 * g_i (i != 0) as deviations from w_i times an equilibrium reference. */
enum pflbm_precision { PFLBM_FP64 = 0, PFLBM_FP32 = 1, PFLBM_BF16 = 2, PFLBM_FP16 = 3 };

/* Node classes (Sec. 2.2.2-2.2.3): fluid (zeta = 1, epsilon = 1); boundary =
 * solid with a non-solid 8-neighbour (zeta = 1, epsilon = 0: collides and
 * streams, bounce-back); ghost = other solid with a zeta = 1 neighbour
 * (zeta = 0, phi = zeta-weighted neighbour mean); interior = other solid. */
enum pflbm_node_class { PFLBM_FLUID = 0, PFLBM_BOUNDARY = 1, PFLBM_GHOST = 2, PFLBM_INTERIOR = 3 };

typedef struct {
    int nx, ny;
    const uint8_t* solid_mask;     /* [ny][nx], 1 = solid; copied             */
    double theta_deg;              /* uniform contact angle (degrees)         */
    const float* theta_field_deg;  /* optional [ny][nx] angle field; copied   */
    double sigma, W, M, tau_f, rho_l, rho_g;
    double tau_g;                  /* <= 0: 1.0                               */
    int precision;                 /* enum pflbm_precision                    */
    int device;                    /* CUDA ordinal; < 0: the current device   */
    void* stream;                  /* cudaStream_t; NULL: a stream created and
                                      owned by the handle                     */
    /* Optional device allocator (e.g. a framework's caching allocator).
     * Both NULL: cudaMalloc / cudaFree. alloc returns NULL on failure. */
    void* (*alloc)(size_t bytes, void* ctx);
    void (*free)(void* ptr, size_t bytes, void* ctx);
    void* alloc_ctx;
    /* Variable viscosity (Sec. 2.1.1): nu(phi) = phi (nu_l - nu_g) + nu_g,
     * tau_f(x) = nu(phi(x)) / c_s^2 + 1/2 (Sec. 2.1.2) at every node. Used
     * when both are > 0; otherwise the uniform tau_f above. */
    double nu_l, nu_g;
    /* Body force F_b = rho g (Sec. 2.1.1, F = F_s + F_b in Eq. GGi):
     * a uniform acceleration (gx, gy); 0 by default. */
    double gx, gy;
    /* The (1/2) dt^2 dG_i/dt term of Eq. BGK: 0 = backward difference
     * (1/2)[G_i(t) - G_i(t-1)] (default); 1 = omitted, source G_i(t) only
     * (no u.grad(phi) history is read or written). The paper does not say
     * how the derivative is discretised; the backward difference lets
     * period-2-in-time modes grow after ~2e4 steps in some cases. */
    int dgdt_mode;
    /* Appendix A, Table 2 (0 or 2: case 2, the paper's method). Cases 1
     * and 3 move the wall energy into a Robin ghost condition
     * n_w . grad(phi) = chi = -/+ sqrt(2 beta/kappa) cos(theta) (phi - phi^2)
     * on flat walls (the ghost's mirror is the zeta = 1 node straight above
     * or below; other ghosts keep the mean), with mu carrying the a_v wall
     * term 0 times (case 1) or twice (case 3). */
    int chi_case;
    /* Step kernel (results are identical bit for bit; only the speed
     * differs). 0: the library's default, by the measured crossover: 4 for
     * 16-bit storage on lattices of at least 2^19 nodes and for FP32 on
     * lattices of at least 2^21 nodes, else 1;
     * 1: populations pulled from global memory, 32 x 8 tiles; 2:
     * populations staged in shared memory by TMA, 32 x 8 tiles; 3: staged,
     * 64 x 4 tiles; 4: global loads, two x-adjacent nodes per thread in
     * packed FP32x2 arithmetic, 64 x 8 tiles. FP64 handles always use 1.
     * step_chunk: tiles a CTA of the staged kernel marches down one tile
     * column per work item (<= 0: 16). */
    int step_kernel;
    int step_chunk;
} pflbm_params_t;

/* Flat, inclined or circular wall for the contact-angle fit. type 0: the
 * straight wall through (px, py) with unit normal (nx, ny) pointing into the
 * fluid; type 1: a circular solid of centre (px, py) and radius r. Only the
 * phi = 1/2 crossings between fluid nodes with x_lo <= x < x_hi and farther
 * than `exclude` from the wall are fitted. */
typedef struct {
    int type;
    double px, py, nx, ny, r;
    double x_lo, x_hi;
    double exclude;
} pflbm_wall_t;

/* Fill p with defaults: theta 90, sigma 0.01, W 4, M 0.1, tau_f 0.8,
 * rho_l 1, rho_g 0.1, tau_g 1, FP32, current device, own stream. */
void pflbm_params_default(pflbm_params_t* p);

/* Create a solver from the problem statement of Sec. 3 (lattice, solid mask,
 * theta, sigma, W, M, tau_f, rho_l, rho_g), FP32 storage. Classifies the
 * nodes and computes a_v = |grad epsilon| (Eq. avvv) on the device.
 * Errors: EINVAL (sizes: nx >= 3, 5 <= ny <= 524280, 18 ny pitch < 2^31 with
 * pitch = nx rounded up to 64; parameters: W > 0, M > 0, tau_f > 1/2,
 * densities > 0, sigma >= 0), EBADMASK, ENOMEM, ECUDA. *out is NULL on
 * failure. */
int pflbm_create(pflbm_t** out, int nx, int ny, const uint8_t* solid_mask, double theta_deg,
                 double sigma, double W, double M, double tau_f, double rho_l, double rho_g);
/* Same with every option (precision, tau_g, angle field, device, stream,
 * allocator). */
int pflbm_create_ex(pflbm_t** out, const pflbm_params_t* p);
/* Release every device buffer of the handle (NULL is ignored). */
void pflbm_destroy(pflbm_t* h);

/* Switch the step kernel of a handle (values as pflbm_params_t.step_kernel
 * and step_chunk). EINVAL for a staged kernel on an FP64 handle or when the
 * handle's tensor maps could not be built. */
int pflbm_set_step_kernel(pflbm_t* h, int step_kernel, int step_chunk);
/* The step kernel a handle uses (1 to 4 as above). */
int pflbm_get_step_kernel(const pflbm_t* h);

/* Replace the contact-angle field (degrees, [ny][nx], copied). Takes effect
 * from the next step. */
int pflbm_set_theta_field(pflbm_t* h, const float* theta_deg);

/* Initial droplet of Eq. initialphi, phi = 1/2 + 1/2 tanh(2 (R - r) / W)
 * with r the x-periodic distance to (x0, y0). The first call after create or
 * after a step replaces phi; further calls keep the pointwise maximum. Sets
 * u = 0, p = 0 (f_i = 0) and g_i = g_i^eq(phi, mu) (Eq. H_i). The profile
 * and mu are evaluated in FP64 for PFLBM_FP64 handles, in FP32 otherwise
 * (r itself in FP64); beyond r = |R| + 10 W phi is 0. Asynchronous. */
int pflbm_init_droplet(pflbm_t* h, double x0, double y0, double R);
/* General initial field phi [ny][nx] (host, copied; values on zeta = 0 nodes
 * are ignored); same initial populations as above. */
int pflbm_init_phi(pflbm_t* h, const double* phi);

/* n time steps (Eqs. BGK-NS, BGK with the chemical potential of Eq.
 * chemical_potencial2, streaming and modified bounce-back, Sec. 2.2.2).
 * Asynchronous on the handle's stream; returns ENUMERIC if an earlier step
 * reported a NaN or |u| >= 0.3 (the flag is read back without blocking). */
int pflbm_step(pflbm_t* h, int64_t n);

/* Macroscopic fields of the current state (synchronous). phi [ny][nx] (ghost
 * nodes: the ghost average; interior nodes: 0), u [ny][nx][2] (ux, uy),
 * p [ny][nx] (u = p = 0 on zeta = 0 nodes). Any pointer may be NULL.
 * Caller-owned host buffers. */
int pflbm_get(pflbm_t* h, double* phi, double* u, double* p);
/* The same fields rounded to float (round to nearest), for callers that
 * read back FP32 or 16-bit solves: half the bytes of pflbm_get. */
int pflbm_get_f32(pflbm_t* h, float* phi, float* u, float* p);
/* Same into caller-owned DEVICE buffers (no host copy, asynchronous). */
int pflbm_get_device(pflbm_t* h, double* phi, double* u, double* p);

/* FP64 sum of phi = sum_i g_i over zeta = 1 nodes (synchronous). */
int pflbm_mass(pflbm_t* h, double* out);

/* FP64 sum of a phi field held in caller-owned DEVICE memory, over the nodes
 * with d_zeta[k] != 0 (every node when d_zeta is NULL): the mass reduction of
 * pflbm_mass applied to, e.g., the phi written by pflbm_get_device. The paper
 * has no counterpart; this entry point exists for callers that cannot
 * allocate device memory (a component inside a framework whose pool owns the
 * device, or a loop where cudaMalloc's possible device synchronisation is not
 * allowed) and so cannot create a handle. It allocates nothing: its block
 * partials live in a static 32 KB device array that the library holds on
 * every GPU it is loaded on until exit. d_phi: [ny][nx] doubles; d_zeta:
 * [ny][nx] bytes or NULL; d_out: one double, written asynchronously on
 * `stream` (cudaStream_t, NULL = default stream) of the current device.
 * The first call on a device looks up the array's device address; make that
 * first call before any stream capture. The address is kept per CUDA context:
 * after cudaDeviceReset the next call looks it up again, so it too belongs
 * before any capture. Calls whose kernels overlap on the
 * GPU share the array and race. Errors: EINVAL for NULL phi/out, nx or
 * ny < 1, or nx * ny > 33,554,432 (the static limit); ECUDA. */
int pflbm_phi_mass_noalloc(const double* d_phi, const uint8_t* d_zeta, int nx, int ny, double* d_out,
                           void* stream);

/* Contact angle (degrees) from a circle fitted to the phi = 1/2 crossings,
 * measured through the liquid against the given wall (synchronous; FP64 on
 * the device). circle (may be NULL) receives {centre x, centre y, R};
 * npoints (may be NULL) the number of fitted points. EINVAL if fewer than
 * 3 points. */
int pflbm_contact_angle(pflbm_t* h, const pflbm_wall_t* wall, double* theta_deg, double* circle,
                        int* npoints);

/* Geometry read-back (synchronous): node class, unknown-link mask (bit i set
 * when zeta(x - c_i) = 0 at a zeta = 1 node), doubly-unknown mask (also
 * zeta(x + c_i) = 0), a_v. Any pointer may be NULL. Bit order: the library's
 * velocity order from pflbm_lattice. */
int pflbm_geometry(pflbm_t* h, uint8_t* cls, uint16_t* unknown, uint16_t* doubly, double* av);
/* The library's D2Q9 velocity order (cx[i], cy[i], i = 0..8). */
void pflbm_lattice(int cx[9], int cy[9]);

/* Synchronise the handle's stream and report ENUMERIC / ECUDA if any. */
int pflbm_check(pflbm_t* h);
/* The status last copied back from the device, without waiting: PFLBM_OK or
 * PFLBM_ENUMERIC (may lag the device by the steps still in flight). */
int pflbm_status(const pflbm_t* h);
/* Steps taken since the last initialisation. */
int64_t pflbm_steps(const pflbm_t* h);

/* Device bytes a handle of this size and precision allocates. */
size_t pflbm_footprint_bytes(int nx, int ny, int precision);

/* Checkpoint: *len in: capacity of buf, out: bytes needed/written. buf may be
 * NULL to query the size. The blob holds the populations, the u.grad(phi)
 * history, the step count, the parameters and flags (derived beta, kappa,
 * alpha, tau_f, tau_g, rho_l, rho_g, W, sigma, M; nu_l, nu_g, gx, gy;
 * dgdt_mode, chi_case) and a 64-bit fingerprint of the node bytes and
 * wetting coefficients (so of the solid mask and the angle field where it
 * acts). Load requires a handle of the same size and precision whose
 * parameters, flags and fingerprint are equal; otherwise PFLBM_EINVAL and the
 * handle is unchanged. Both synchronous. */
int pflbm_save(pflbm_t* h, void* buf, size_t* len);
int pflbm_load(pflbm_t* h, const void* buf, size_t len);

/* ---- many lattices per launch ------------------------------------------
 * A batch advances several handles (of any sizes) together: each time step
 * is one persistent launch over a work list of (lattice, tile) items (or,
 * with kernel 3, one launch per group of same-size lattices), and runs of 8
 * steps can be replayed from a captured CUDA graph. The per-node
 * update is exactly that of pflbm_step; the paper has no batching. All
 * handles of a batch must share precision, device and stream; the batch runs
 * on that stream and keeps no copy of the handles' state. */
typedef struct pflbm_batch pflbm_batch_t;
typedef struct {
    int ctas_per_sm;     /* persistent CTAs per SM; <= 0: as many as fit      */
    int tiles_per_item;  /* tiles of one tile column per work item (lattices
                            no size class below covers)                       */
    int order;           /* 0: lattice by lattice; 1: largest lattices first,
                            items interleaved across lattices                 */
    int use_graph;       /* replay runs of 8 steps from a captured CUDA graph */
    int kernel;          /* 0: default (3); 1: global-load kernel, 32 x 8
                            tiles; 2: staged kernel (TMA ring) with the
                            size classes below; 3: two-node kernel (two
                            x-adjacent nodes per thread in packed FP32x2
                            arithmetic), one launch per group of lattices
                            of one size, one 64 x 8 tile per CTA, the
                            groups' launches side by side (tiles_per_item,
                            order and ctas_per_sm do not apply). FP64
                            batches always use 1.                           */
    /* Staged kernel, per size class: a lattice with nx * ny <=
     * class_max_nodes[k] (first such k < n_classes) runs with tile shape
     * class_shape[k] (0: 32 x 8, 1: 64 x 4) and class_tiles[k] tiles per
     * work item; other lattices with 32 x 8 and tiles_per_item. */
    int n_classes;
    int64_t class_max_nodes[8];
    int class_shape[8];
    int class_tiles[8];
} pflbm_schedule_t;

/* Defaults: as many CTAs as fit, 1 tile per item, order 0, graphs on,
 * default kernel, no size classes. */
void pflbm_schedule_default(pflbm_schedule_t* s);
/* Build a batch over hs[0..count-1] (schedule NULL: defaults). Allocates the
 * device work list and descriptors with cudaMalloc. EINVAL if the handles
 * differ in precision, device or stream, or repeat. Members may be destroyed
 * while the batch lives, as long as pflbm_batch_set drops them before the
 * next pflbm_batch_step. */
int pflbm_batch_create(pflbm_batch_t** out, pflbm_t* const* hs, int count, const pflbm_schedule_t* sched);
/* Replace the members (same rules); reuses the device buffers when they are
 * large enough. */
int pflbm_batch_set(pflbm_batch_t* b, pflbm_t* const* hs, int count);
/* n time steps of every member (asynchronous). Members stepped on their own
 * in between are picked up (descriptors are rewritten). ENUMERIC if a member
 * reported a NaN or |u| >= 0.3 earlier. */
int pflbm_batch_step(pflbm_batch_t* b, int64_t n);
/* The step kernel the batch runs (1 global loads, 2 staged, 3 two-node). */
int pflbm_batch_kernel(const pflbm_batch_t* b);
/* Work items, persistent grid size and total nodes of the batch (kernel 3:
 * the CTAs of all launches, one 64 x 8 tile each, and the number of
 * launches per step). */
int pflbm_batch_info(const pflbm_batch_t* b, int* n_work, int* grid, int64_t* nodes);
void pflbm_batch_destroy(pflbm_batch_t* b);

/* Index-checked debug build (compiled with -DPFLBM_BOUNDS, shipped as
 * libpflbm_bounds.so beside the library): every global and staged
 * shared-memory index of the 2D step kernels is checked against its buffer;
 * an index outside is counted and the access skipped. *enabled: 1 in that
 * build, 0 in the normal one; *violations: accesses refused so far on the
 * current device (0 in the normal build). Not in the paper: a test aid. */
int pflbm_debug_bounds(int* enabled, unsigned* violations);

/* Text of the calling thread's last error ("" if none). */
const char* pflbm_last_error(void);

/* ------------------------------------------------------------------------
 * Three dimensions (Sec. 2.1.2-2.1.3 and 2.2.2 with their 3D lattices): f on
 * D3Q19 (w = 1/3, 1/18, 1/36, c_s^2 = 1/3), g on D3Q7 (the paper's velocity
 * matrix, w = 1/4, 1/8, c_s^2 = 1/4, so alpha = M / (c_s^2 (tau_g - 1/2))
 * takes 1/4), gradients, Laplacian and a_v = |grad epsilon| with the D3Q19
 * weights, and the ghost value as the zeta-weighted mean of the 27
 * surrounding nodes (b = 27).
 *
 * Fields are [nz][ny][nx], node (x, y, z) at (z*ny + y)*nx + x. x and y are
 * periodic; planes z = 0, 1, nz-2 and nz-1 must be solid. Velocity orders:
 * D3Q19 rest, +x, -x, +y, -y, +z, -z, then (+x+y, -x-y, +x-y, -x+y, +x+z,
 * -x-z, +x-z, -x+z, +y+z, -y-z, +y-z, -y+z); D3Q7 is the first seven.
 * Classes as in 2D with the 18-neighbourhood of D3Q19 for "neighbour".
 * Precision: PFLBM_FP64 or PFLBM_FP32 (g_0 in 32-bit fixed point as in 2D).
 * The library allocates its device memory with cudaMalloc, or with the
 * allocator callbacks of pflbm3d_params_t when they are set; the state takes
 * 2 x 26 population planes of nz*ny*pitch elements (pitch = nx rounded up to
 * 64) plus 8 further planes. Sizes: nx, ny >= 3, 5 <= nz <= 65535,
 * ny <= 524280, 26 nz ny pitch < 2^31 (EINVAL otherwise). Error behaviour as
 * for the 2D calls.
 * ------------------------------------------------------------------------ */
typedef struct pflbm3d pflbm3d_t;

typedef struct {
    int nx, ny, nz;
    const uint8_t* solid_mask;   /* [nz][ny][nx], nonzero = solid; copied */
    double theta_deg, sigma, W, M, tau_f, rho_l, rho_g;
    double tau_g;                /* <= 0: 1 */
    int precision;               /* PFLBM_FP64 or PFLBM_FP32 */
    int device;                  /* CUDA device; < 0: current */
    void* stream;                /* cudaStream_t; NULL: a stream of its own */
    int step_path;               /* enum pflbm3d_step_path; the results are identical */
    int fused_zc;                /* planes per CTA of the fused step; <= 0: chosen by the library */
    int dgdt_mode;               /* as pflbm_params_t.dgdt_mode: 0 backward difference, 1 omitted */
    /* Optional device allocator, as in pflbm_params_t (both NULL: cudaMalloc /
     * cudaFree). Every buffer is returned through free at pflbm3d_destroy. */
    void* (*alloc)(size_t bytes, void* ctx);
    void (*free)(void* ptr, size_t bytes, void* ctx);
    void* alloc_ctx;
} pflbm3d_params_t;

/* How a 3D step runs. PFLBM3D_FUSED: one launch; each CTA marches a 32 x 8
 * column through z, recomputing phi and the ghost values of its halo in
 * shared memory. PFLBM3D_THREE_PASS: phi, ghost values and the
 * collide-and-store as three launches through a phi array in HBM.
 * PFLBM3D_AUTO (0): the faster of the two on GB300 (three launches). */
enum pflbm3d_step_path { PFLBM3D_AUTO = 0, PFLBM3D_FUSED = 1, PFLBM3D_THREE_PASS = 2 };

void pflbm3d_params_default(pflbm3d_params_t* p);
int pflbm3d_create(pflbm3d_t** out, const pflbm3d_params_t* p);
void pflbm3d_destroy(pflbm3d_t* h);
/* Initial field: tanh sphere of radius R centred at (x0, y0, z0) (Eq.
 * initialphi), periodic in x and y; the first call after creation or a step
 * replaces the field, later calls take the maximum. Precision and reach as
 * for pflbm_init_droplet. */
int pflbm3d_init_droplet(pflbm3d_t* h, double x0, double y0, double z0, double R);
/* Initial field from a host array [nz][ny][nx] (values on zeta = 0 nodes are
 * ignored). */
int pflbm3d_init_phi(pflbm3d_t* h, const double* phi);
/* n time steps on the handle's stream (asynchronous). */
int pflbm3d_step(pflbm3d_t* h, int64_t n);
/* phi [N] (ghost values on ghost nodes, 0 inside the solid), u [N][3] and p
 * [N] (0 off zeta = 1 nodes) into host arrays; any may be NULL. Synchronous. */
int pflbm3d_get(pflbm3d_t* h, double* phi, double* u, double* p);
/* The same fields rounded to float (round to nearest): half the bytes. */
int pflbm3d_get_f32(pflbm3d_t* h, float* phi, float* u, float* p);
/* sum of the g_i over zeta = 1 nodes, FP64, fixed order. Synchronous. */
int pflbm3d_mass(pflbm3d_t* h, double* out);
/* node classes (pflbm_node_class) and a_v into host arrays [N]; either may
 * be NULL. Synchronous. */
int pflbm3d_geometry(pflbm3d_t* h, uint8_t* cls, double* av);
/* Waits for the stream; PFLBM_ENUMERIC if a NaN or |u| >= 0.3 was seen. */
int pflbm3d_check(pflbm3d_t* h);
/* Steps taken since the last initialisation (-1 for a NULL handle). */
int64_t pflbm3d_steps(const pflbm3d_t* h);
/* Checkpoint of the state (populations, u.grad(phi) history, step count,
 * the derived parameters, dgdt_mode and a fingerprint of the node bytes and
 * wetting coefficients) into a caller buffer; buf == NULL returns the size in
 * *len. pflbm3d_load restores it into a handle of the same size, precision,
 * parameters and geometry, after which the steps continue bit for bit as if
 * uninterrupted. Synchronous. Errors: EINVAL (buffer too small, not a
 * checkpoint, or any of those differs; the handle is then unchanged). */
int pflbm3d_save(pflbm3d_t* h, void* buf, size_t* len);
int pflbm3d_load(pflbm3d_t* h, const void* buf, size_t len);

/* Wall for the 3D contact-angle fit. type 0: the plane through (px, py, pz)
 * with unit normal (nx, ny, nz) pointing into the fluid; type 1: a solid
 * sphere of centre (px, py, pz) and radius r. Only the crossings with
 * x_lo <= x < x_hi, y_lo <= y < y_hi and farther than `exclude` from the wall
 * are fitted (the window separates droplets of a many-droplet lattice). */
typedef struct {
    int type;
    double px, py, pz, nx, ny, nz, r;
    double x_lo, x_hi, y_lo, y_hi;
    double exclude;
} pflbm3d_wall_t;

/* Contact angle of one droplet (the 3D form of the fits of Secs. 3.1-3.3),
 * in FP64 on the device: the phi = 1/2 crossings between fluid neighbours, a
 * sphere fit, and theta from cos(theta) = -n.(c - p)/R (plane) or
 * (R^2 + r^2 - |c - p|^2)/(2 R r) (sphere). theta is NaN when fewer than 4
 * points remain. sphere (optional, 4 doubles) receives the fitted centre and
 * radius, npoints (optional) the point count. The first call allocates a
 * point buffer of min(3 N, 2^22) points. Synchronous. Errors: EINVAL,
 * ENOMEM, ECUDA. */
int pflbm3d_contact_angle(pflbm3d_t* h, const pflbm3d_wall_t* wall, double* theta_deg, double* sphere,
                          int* npoints);

#ifdef __cplusplus
}
#endif
#endif /* PFLBM_H */
