// capi.cu -- the extern "C" entry points of libpflbm.so (declared and
// documented in include/pflbm.h): argument checks, device memory, streams,
// error codes. Every computation runs in the kernels of geometry.cu, step.cu
// and diag.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "storage.cuh"

namespace pfk {
size_t mass_scratch_doubles();
}

using namespace pfk;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg)
{
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* where)
{
    return fail(PFLBM_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                          \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

int dalloc(pflbm_t* h, void** p, size_t bytes)
{
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (h->alloc_fn) {
        *p = h->alloc_fn(bytes, h->alloc_ctx);
        if (!*p) return fail(PFLBM_ENOMEM, "allocator callback returned NULL");
    } else {
        cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            *p = nullptr;
            return fail(PFLBM_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
    }
    h->bytes_allocated += bytes;
    return PFLBM_OK;
}

void dfree(pflbm_t* h, void* p, size_t bytes)
{
    if (!p) return;
    if (h->free_fn)
        h->free_fn(p, bytes, h->alloc_ctx);
    else
        cudaFree(p);
}

int pitch_of(int nx) { return (nx + 63) / 64 * 64; }

struct Sizes {
    size_t N, pop, sprev, wet, red, pts, tiles;
    int pts_cap;
};

Sizes sizes_of(int nx, int ny, int precision)
{
    Sizes s{};
    int pitch = pitch_of(nx);
    s.N = (size_t)ny * pitch;
    s.pop = pop_bytes(ny, pitch, precision);
    size_t cs = precision == PFLBM_FP64 ? 8 : 4;
    s.sprev = s.N * cs;
    s.wet = s.N * cs;
    s.red = mass_scratch_doubles() * sizeof(double);
    long long cap = 2LL * nx * ny;
    if (cap > (1 << 22)) cap = 1 << 22;
    s.pts_cap = (int)cap;
    s.pts = (size_t)s.pts_cap * 2 * sizeof(double);
    s.tiles = (size_t)tiles_x(nx) * tiles_y(ny);
    return s;
}

bool valid_params(const pflbm_params_t* p, std::string& why)
{
    if (p->nx < 3 || p->ny < 5) { why = "nx must be >= 3 and ny >= 5"; return false; }
    if ((p->ny + TY - 1) / TY > 65535) {
        why = "ny too large (at most 524280 rows: one launch row of tiles per 8 rows)";
        return false;
    }
    if (18LL * p->ny * ((p->nx + 63) / 64 * 64) >= (1LL << 31)) {
        why = "lattice too large (18 * ny * padded nx must stay below 2^31)";
        return false;
    }
    if (!p->solid_mask) { why = "solid_mask is NULL"; return false; }
    if (!(p->W > 0) || !(p->M > 0) || !(p->tau_f > 0.5) || !(p->rho_l > 0) || !(p->rho_g > 0) ||
        !(p->sigma >= 0) || !std::isfinite(p->theta_deg)) {
        why = "need W > 0, M > 0, tau_f > 1/2, rho_l > 0, rho_g > 0, sigma >= 0, finite theta";
        return false;
    }
    if (p->tau_g > 0 && !(p->tau_g > 0.5)) { why = "tau_g must be > 1/2"; return false; }
    if (!std::isfinite(p->nu_l) || !std::isfinite(p->nu_g) || !std::isfinite(p->gx) || !std::isfinite(p->gy) ||
        p->nu_l < 0 || p->nu_g < 0) {
        why = "nu_l, nu_g must be finite and >= 0; gx, gy finite";
        return false;
    }
    if (p->dgdt_mode != 0 && p->dgdt_mode != 1) { why = "dgdt_mode must be 0 or 1"; return false; }
    if (p->chi_case < 0 || p->chi_case > 3) { why = "chi_case must be 1, 2 or 3 (0: 2)"; return false; }
    if (p->precision < PFLBM_FP64 || p->precision > PFLBM_FP16) {
        why = "precision must be PFLBM_FP64, PFLBM_FP32, PFLBM_BF16 or PFLBM_FP16";
        return false;
    }
    if ((p->alloc == nullptr) != (p->free == nullptr)) { why = "alloc and free must be given together"; return false; }
    return true;
}

void release(pflbm_t* h)
{
    if (!h) return;
    Sizes s = sizes_of(h->nx, h->ny, h->precision);
    DeviceGuard g(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    dfree(h, h->cls, s.N);
    dfree(h, h->tiles, s.tiles);
    dfree(h, h->solid, s.N);
    dfree(h, h->theta, s.N * sizeof(float));
    dfree(h, h->wet, s.wet);
    dfree(h, h->av, s.N * sizeof(double));
    dfree(h, h->pop[0], s.pop);
    dfree(h, h->pop[1], s.pop);
    dfree(h, h->sprev, s.sprev);
    dfree(h, h->phi0, s.N * sizeof(double));
    dfree(h, h->mu0, s.N * sizeof(double));
    dfree(h, h->red, s.red);
    dfree(h, h->pts, s.pts);
    dfree(h, h->out, h->out_bytes);
    if (h->out_f) dfree(h, h->out_f, (size_t)h->nx * h->ny * 4 * sizeof(float));
    dfree(h, h->dstatus, sizeof(int) * 4);
    dfree(h, h->tma, tma_sets_bytes());
    dfree(h, h->sflags, staged_flags_bytes(h->nx, h->ny));
    dfree(h, h->nword, node_words_bytes(h->nx, h->ny));
    dfree(h, h->tiles2, tile2_flags_bytes(h->nx, h->ny));
    if (h->hstatus) cudaFreeHost(h->hstatus);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

int check_handle(const pflbm_t* h)
{
    if (!h) return fail(PFLBM_EINVAL, "NULL handle");
    return PFLBM_OK;
}

int read_status(pflbm_t* h)
{
    if (h->hstatus && (h->hstatus[0] & 4))
        return fail(PFLBM_ETIMEOUT, "a wait for staged data in the step kernel gave up");
    if (h->hstatus && h->hstatus[0] != 0) {
        return fail(PFLBM_ENUMERIC, "NaN or |u| >= 0.3 detected on the device");
    }
    return PFLBM_OK;
}

int post_status_copy(pflbm_t* h)
{
    CK(cudaMemcpyAsync(h->hstatus, h->dstatus, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    return PFLBM_OK;
}

// Build the populations from phi0 once after one or more initialisations.
int materialize(pflbm_t* h)
{
    if (!h->init_pending) return PFLBM_OK;
    CK(launch_init_populations(h));
    CK(cudaMemsetAsync(h->dstatus, 0, sizeof(int), h->stream));
    if (h->hstatus) h->hstatus[0] = 0;
    h->init_pending = false;
    return PFLBM_OK;
}

int ensure_out(pflbm_t* h)
{
    if (h->out) return PFLBM_OK;
    size_t bytes = (size_t)h->nx * h->ny * 4 * sizeof(double);
    void* p = nullptr;
    int rc = dalloc(h, &p, bytes);
    if (rc) return rc;
    h->out = (double*)p;
    h->out_bytes = bytes;
    return PFLBM_OK;
}

// Step kernel of a handle (pflbm_params_t.step_kernel). 0 picks the default
// by storage and lattice size, from the measured crossover on lattices of 5k
// to 8.4M nodes (warm, MLUPS):
// - 16-bit storage: the two-node kernel from 2^19 nodes (6 to 32 % faster
//   there; 5 to 25 % slower at 2^18 nodes and below);
// - FP32: the two-node kernel from 2^21 nodes (2 to 4 % faster there; within
//   0.5 % at 2^20 nodes, 0.2 to 25 % slower at 2^19 nodes and below);
// - otherwise, and for FP64, the one-node global-load kernel: its 32 x 8
//   tiles give a small lattice twice the CTAs, and each CTA does half the
//   work. The staged kernel was slower on every workload (about 6 % more
//   instructions per node, 4 instead of 6 resident CTAs per SM).
constexpr long long kPairMinNodes16 = 1LL << 19, kPairMinNodes32 = 1LL << 21;

int select_step_kernel(pflbm_t* h, int kernel, int chunk)
{
    if (kernel < 0 || kernel > 4) return fail(PFLBM_EINVAL, "step_kernel must be 0, 1, 2, 3 or 4");
    if (kernel == 0) {
        const long long nodes = (long long)h->nx * h->ny;
        const bool b16 = h->precision == PFLBM_BF16 || h->precision == PFLBM_FP16;
        kernel = (b16 && nodes >= kPairMinNodes16) || (h->precision == PFLBM_FP32 && nodes >= kPairMinNodes32) ? 4 : 1;
    }
    if (kernel == 4) {
        if (h->precision == PFLBM_FP64) return fail(PFLBM_EINVAL, "the two-node step kernel needs FP32 or 16-bit storage");
        h->step_shape = -2;
        h->step_chunk = chunk > 0 ? chunk : 16;
        return PFLBM_OK;
    }
    if (kernel >= 2 && (h->precision == PFLBM_FP64 || !h->tma))
        return fail(PFLBM_EINVAL, "the staged step kernel needs FP32 or 16-bit storage and its tensor maps");
    h->step_shape = kernel - 2;
    h->step_chunk = chunk > 0 ? chunk : 16;
    return PFLBM_OK;
}

// Sets *flag when a value of the [ny][pitch] angle field (first nx columns)
// is not finite.
__global__ void k_theta_finite(const float* __restrict__ theta, int nx, int ny, int pitch, int* flag)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x < nx && y < ny && !isfinite(theta[(size_t)y * pitch + x])) atomicOr(flag, 1);
}

}  // namespace

namespace pfk {
int set_error(int code, const char* msg) { return fail(code, msg); }
int materialize_handle(pflbm_t* h) { return materialize(h); }
int post_status(pflbm_t* h) { return post_status_copy(h); }

size_t elem_size(int precision)
{
    switch (precision) {
        case PFLBM_FP64: return 8;
        case PFLBM_FP32: return 4;
        default: return 2;
    }
}
size_t pop_bytes(int ny, int pitch, int precision) { return state_copy_bytes(precision, (size_t)ny * pitch); }
}  // namespace pfk

extern "C" {

void pflbm_params_default(pflbm_params_t* p)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->theta_deg = 90.0;
    p->sigma = 0.01;
    p->W = 4.0;
    p->M = 0.1;
    p->tau_f = 0.8;
    p->rho_l = 1.0;
    p->rho_g = 0.1;
    p->tau_g = 1.0;
    p->precision = PFLBM_FP32;
    p->device = -1;
}

void pflbm_lattice(int cxo[9], int cyo[9])
{
    for (int i = 0; i < 9; ++i) {
        if (cxo) cxo[i] = cx(i);
        if (cyo) cyo[i] = cy(i);
    }
}

const char* pflbm_last_error(void) { return g_last_error.c_str(); }

size_t pflbm_footprint_bytes(int nx, int ny, int precision)
{
    if (nx < 1 || ny < 1) return 0;
    Sizes s = sizes_of(nx, ny, precision);
    return 2 * s.pop + s.sprev + s.wet + s.N * (1 + 1 + 8 + 8 + 8) + s.red + s.pts + s.tiles + 16 +
           (size_t)nx * ny * 4 * sizeof(double) +
           (precision != PFLBM_FP64 ? tma_sets_bytes() + staged_flags_bytes(nx, ny) + node_words_bytes(nx, ny) +
                                          tile2_flags_bytes(nx, ny)
                                    : 0);
}

int pflbm_create_ex(pflbm_t** out, const pflbm_params_t* prm)
{
    if (!out || !prm) return fail(PFLBM_EINVAL, "NULL argument");
    *out = nullptr;
    std::string why;
    if (!valid_params(prm, why)) return fail(PFLBM_EINVAL, why);
    const int nx = prm->nx, ny = prm->ny;
    for (int x = 0; x < nx; ++x) {
        if (!prm->solid_mask[x] || !prm->solid_mask[nx + x] || !prm->solid_mask[(size_t)(ny - 2) * nx + x] ||
            !prm->solid_mask[(size_t)(ny - 1) * nx + x])
            return fail(PFLBM_EBADMASK, "rows 0, 1, ny-2 and ny-1 of the solid mask must be solid");
    }
    // a non-finite value in the angle field is found on the device, after the copy
    pflbm_t* h = new (std::nothrow) pflbm();
    if (!h) return fail(PFLBM_ENOMEM, "host allocation failed");
    h->nx = nx;
    h->ny = ny;
    h->pitch = pitch_of(nx);
    h->precision = prm->precision;
    h->alloc_fn = prm->alloc;
    h->free_fn = prm->free;
    h->alloc_ctx = prm->alloc_ctx;
    h->theta_uniform = prm->theta_deg;
    int dev = prm->device;
    if (dev < 0) {
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) { delete h; return cuda_fail(e, "cudaGetDevice"); }
    }
    h->device = dev;
    DeviceGuard guard(dev);
    // derived parameters (Eqs. b1, initialphi, mobility)
    Params& q = h->prm;
    q.sigma = prm->sigma;
    q.W = prm->W;
    q.M = prm->M;
    q.beta = 12.0 * prm->sigma / prm->W;
    q.kappa = 1.5 * prm->sigma * prm->W;
    q.tau_f = prm->tau_f;
    q.tau_g = prm->tau_g > 0 ? prm->tau_g : 1.0;
    q.alpha = prm->M / ((1.0 / 3.0) * (q.tau_g - 0.5));
    q.rho_l = prm->rho_l;
    q.rho_g = prm->rho_g;
    q.nu_l = (prm->nu_l > 0 && prm->nu_g > 0) ? prm->nu_l : 0.0;
    q.nu_g = (prm->nu_l > 0 && prm->nu_g > 0) ? prm->nu_g : 0.0;
    q.gx = prm->gx;
    q.gy = prm->gy;
    q.dgdt_mode = prm->dgdt_mode;
    q.chi_case = prm->chi_case == 0 ? 2 : prm->chi_case;

    if (prm->stream) {
        h->stream = (cudaStream_t)prm->stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete h; return cuda_fail(e, "cudaStreamCreate"); }
        h->own_stream = true;
    }
    Sizes s = sizes_of(nx, ny, h->precision);
    int rc = PFLBM_OK;
    void* p;
#define ALLOC(field, bytes)                                   \
    do {                                                      \
        rc = dalloc(h, &p, (bytes));                          \
        if (rc) { release(h); return rc; }                    \
        h->field = (decltype(h->field))p;                     \
    } while (0)
    ALLOC(cls, s.N);
    ALLOC(tiles, s.tiles);
    ALLOC(solid, s.N);
    ALLOC(wet, s.wet);
    ALLOC(av, s.N * sizeof(double));
    ALLOC(pop[0], s.pop);
    ALLOC(pop[1], s.pop);
    ALLOC(sprev, s.sprev);
    ALLOC(phi0, s.N * sizeof(double));
    ALLOC(mu0, s.N * sizeof(double));
    ALLOC(red, s.red);
    ALLOC(pts, s.pts);
    ALLOC(dstatus, sizeof(int) * 4);
    if (prm->theta_field_deg) ALLOC(theta, s.N * sizeof(float));
#undef ALLOC
    h->pts_cap = s.pts_cap;
    if (cudaMallocHost((void**)&h->hstatus, sizeof(int) * 4) != cudaSuccess) {
        cudaGetLastError();
        h->hstatus = nullptr;
        release(h);
        return fail(PFLBM_ENOMEM, "cudaMallocHost failed");
    }
    h->hstatus[0] = 0;
    h->hstatus[1] = 0;
#define CKR(call)                                                 \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) { int r_ = cuda_fail(e_, #call); release(h); return r_; } \
    } while (0)
    CKR(cudaMemsetAsync(h->pop[0], 0, s.pop, h->stream));
    CKR(cudaMemsetAsync(h->pop[1], 0, s.pop, h->stream));
    CKR(cudaMemsetAsync(h->sprev, 0, s.sprev, h->stream));
    CKR(cudaMemsetAsync(h->phi0, 0, s.N * sizeof(double), h->stream));
    CKR(cudaMemsetAsync(h->solid, 1, s.N, h->stream));
    CKR(cudaMemsetAsync(h->dstatus, 0, sizeof(int) * 4, h->stream));
    CKR(cudaMemcpy2DAsync(h->solid, h->pitch, prm->solid_mask, nx, nx, ny, cudaMemcpyHostToDevice, h->stream));
    if (prm->theta_field_deg)
        CKR(cudaMemcpy2DAsync(h->theta, h->pitch * sizeof(float), prm->theta_field_deg, nx * sizeof(float),
                              nx * sizeof(float), ny, cudaMemcpyHostToDevice, h->stream));
    if (prm->theta_field_deg) {
        dim3 b(32, 8), g((nx + 31) / 32, (ny + 7) / 8);
        k_theta_finite<<<g, b, 0, h->stream>>>(h->theta, nx, ny, h->pitch, h->dstatus + 1);
        CKR(cudaGetLastError());
        CKR(cudaMemcpyAsync(h->hstatus + 1, h->dstatus + 1, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    }
    CKR(launch_classify(h));
    CKR(launch_tile_flags(h));
    CKR(launch_wet(h));
    // node words and 64 x 8 tile flags of the two-node step (before the
    // tensor maps, which address the node words)
    if (h->precision != PFLBM_FP64) {
        if ((rc = dalloc(h, &p, node_words_bytes(nx, ny)))) { release(h); return rc; }
        h->nword = (uint16_t*)p;
        if ((rc = dalloc(h, &p, tile2_flags_bytes(nx, ny)))) { release(h); return rc; }
        h->tiles2 = (uint8_t*)p;
        CKR(launch_node_words(h));
    }
    // tensor maps of the staged step and of the two-node step's prefetch
    // (FP32 and 16-bit storage)
    std::vector<unsigned char> maps;
    if (h->precision != PFLBM_FP64) {
        maps.resize(tma_sets_bytes() + 64);
        TmaSet* hm = (TmaSet*)(((uintptr_t)maps.data() + 63) & ~(uintptr_t)63);
        if (encode_tma_sets(h, hm)) {
            if ((rc = dalloc(h, &p, tma_sets_bytes()))) { release(h); return rc; }
            h->tma = (TmaSet*)p;
            CKR(cudaMemcpyAsync(h->tma, hm, tma_sets_bytes(), cudaMemcpyHostToDevice, h->stream));
            if ((rc = dalloc(h, &p, staged_flags_bytes(nx, ny)))) { release(h); return rc; }
            h->sflags = (uint8_t*)p;
            CKR(launch_staged_flags(h));
        }
    }
    CKR(cudaStreamSynchronize(h->stream));
#undef CKR
    if (int rc2 = select_step_kernel(h, prm->step_kernel, prm->step_chunk)) {
        release(h);
        return rc2;
    }
    if (prm->theta_field_deg && h->hstatus[1] != 0) {
        release(h);
        return fail(PFLBM_EINVAL, "theta field has a non-finite value");
    }
    *out = h;
    return PFLBM_OK;
}

int pflbm_create(pflbm_t** out, int nx, int ny, const uint8_t* solid_mask, double theta_deg, double sigma,
                 double W, double M, double tau_f, double rho_l, double rho_g)
{
    pflbm_params_t p;
    pflbm_params_default(&p);
    p.nx = nx;
    p.ny = ny;
    p.solid_mask = solid_mask;
    p.theta_deg = theta_deg;
    p.sigma = sigma;
    p.W = W;
    p.M = M;
    p.tau_f = tau_f;
    p.rho_l = rho_l;
    p.rho_g = rho_g;
    return pflbm_create_ex(out, &p);
}

void pflbm_destroy(pflbm_t* h) { release(h); }

int pflbm_debug_bounds(int* enabled, unsigned* violations)
{
#ifdef PFLBM_BOUNDS
    if (enabled) *enabled = 1;
#else
    if (enabled) *enabled = 0;
#endif
    if (violations) *violations = bounds_violations_step() + bounds_violations_tma() + bounds_violations_step2();
    return PFLBM_OK;
}

int pflbm_set_step_kernel(pflbm_t* h, int step_kernel, int step_chunk)
{
    if (int rc = check_handle(h)) return rc;
    return select_step_kernel(h, step_kernel, step_chunk);
}

int pflbm_get_step_kernel(const pflbm_t* h)
{
    if (!h) return PFLBM_EINVAL;
    return h->step_shape == -2 ? 4 : h->step_shape + 2;
}

int pflbm_set_theta_field(pflbm_t* h, const float* theta_deg)
{
    if (int rc = check_handle(h)) return rc;
    if (!theta_deg) return fail(PFLBM_EINVAL, "NULL theta field");
    for (size_t k = 0; k < (size_t)h->nx * h->ny; ++k)
        if (!std::isfinite(theta_deg[k])) return fail(PFLBM_EINVAL, "theta field has a non-finite value");
    DeviceGuard g(h->device);
    if (!h->theta) {
        void* p;
        if (int rc = dalloc(h, &p, (size_t)h->ny * h->pitch * sizeof(float))) return rc;
        h->theta = (float*)p;
    }
    CK(cudaMemcpy2DAsync(h->theta, h->pitch * sizeof(float), theta_deg, h->nx * sizeof(float),
                         h->nx * sizeof(float), h->ny, cudaMemcpyHostToDevice, h->stream));
    CK(launch_wet(h));
    CK(cudaStreamSynchronize(h->stream));
    return PFLBM_OK;
}

int pflbm_init_droplet(pflbm_t* h, double x0, double y0, double R)
{
    if (int rc = check_handle(h)) return rc;
    if (!std::isfinite(x0) || !std::isfinite(y0) || !std::isfinite(R)) return fail(PFLBM_EINVAL, "non-finite droplet");
    DeviceGuard g(h->device);
    CK(launch_init_phi_droplet(h, x0, y0, R, h->replace_phi ? 1 : 0));
    h->replace_phi = false;
    h->init_pending = true;   // populations are built by the next call that needs them
    h->steps = 0;
    return PFLBM_OK;
}

int pflbm_init_phi(pflbm_t* h, const double* phi)
{
    if (int rc = check_handle(h)) return rc;
    if (!phi) return fail(PFLBM_EINVAL, "NULL phi");
    DeviceGuard g(h->device);
    CK(cudaMemcpy2DAsync(h->phi0, h->pitch * sizeof(double), phi, h->nx * sizeof(double), h->nx * sizeof(double),
                         h->ny, cudaMemcpyHostToDevice, h->stream));
    h->replace_phi = false;
    h->init_pending = true;
    CK(cudaStreamSynchronize(h->stream));   // phi is a caller buffer: done with it on return
    h->steps = 0;
    return PFLBM_OK;
}

int pflbm_step(pflbm_t* h, int64_t n)
{
    if (int rc = check_handle(h)) return rc;
    if (n < 0) return fail(PFLBM_EINVAL, "negative step count");
    if (int rc = read_status(h)) return rc;
    DeviceGuard g(h->device);
    NvtxRange range("pflbm_step");
    if (int rc = materialize(h)) return rc;
    for (int64_t t = 0; t < n; ++t) {
        CK(launch_step(h));
        h->steps += 1;
    }
    if (n > 0) {
        h->replace_phi = true;
        if (int rc = post_status_copy(h)) return rc;
    }
    return PFLBM_OK;
}

int pflbm_get_device(pflbm_t* h, double* phi, double* u, double* p)
{
    if (int rc = check_handle(h)) return rc;
    DeviceGuard g(h->device);
    if (int rc = materialize(h)) return rc;
    CK(launch_macro(h, phi, u, p));
    return PFLBM_OK;
}

int pflbm_get(pflbm_t* h, double* phi, double* u, double* p)
{
    if (int rc = check_handle(h)) return rc;
    DeviceGuard g(h->device);
    if (int rc = materialize(h)) return rc;
    if (int rc = ensure_out(h)) return rc;
    size_t N = (size_t)h->nx * h->ny;
    double* dphi = h->out;
    double* du = h->out + N;
    double* dp = h->out + 3 * N;
    CK(launch_macro(h, phi ? dphi : nullptr, u ? du : nullptr, p ? dp : nullptr));
    if (phi) CK(cudaMemcpyAsync(phi, dphi, N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (u) CK(cudaMemcpyAsync(u, du, 2 * N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (p) CK(cudaMemcpyAsync(p, dp, N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return read_status(h);
}

int pflbm_get_f32(pflbm_t* h, float* phi, float* u, float* p)
{
    if (int rc = check_handle(h)) return rc;
    DeviceGuard g(h->device);
    if (int rc = materialize(h)) return rc;
    size_t N = (size_t)h->nx * h->ny;
    if (!h->out_f) {
        void* q = nullptr;
        if (int rc = dalloc(h, &q, 4 * N * sizeof(float))) return rc;
        h->out_f = (float*)q;
    }
    // the read-back kernel writes the float fields directly (phi, u, p at
    // offsets 0, N, 3N): no FP64 scratch
    float* fphi = h->out_f;
    float* fu = h->out_f + N;
    float* fp = h->out_f + 3 * N;
    CK(launch_macro_f32(h, phi ? fphi : nullptr, u ? fu : nullptr, p ? fp : nullptr));
    if (phi) CK(cudaMemcpyAsync(phi, fphi, N * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    if (u) CK(cudaMemcpyAsync(u, fu, 2 * N * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    if (p) CK(cudaMemcpyAsync(p, fp, N * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return read_status(h);
}

int pflbm_mass(pflbm_t* h, double* out)
{
    if (int rc = check_handle(h)) return rc;
    if (!out) return fail(PFLBM_EINVAL, "NULL out");
    DeviceGuard g(h->device);
    if (int rc = materialize(h)) return rc;
    double* d = h->red + mass_scratch_doubles() - 8;
    CK(launch_mass(h, d));
    CK(cudaMemcpyAsync(out, d, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return read_status(h);
}

int pflbm_contact_angle(pflbm_t* h, const pflbm_wall_t* wall, double* theta_deg, double* circle, int* npoints)
{
    if (int rc = check_handle(h)) return rc;
    if (!wall || !theta_deg) return fail(PFLBM_EINVAL, "NULL argument");
    if (wall->type != 0 && wall->type != 1) return fail(PFLBM_EINVAL, "wall type must be 0 or 1");
    if (wall->type == 1 && !(wall->r > 0)) return fail(PFLBM_EINVAL, "circular wall needs r > 0");
    DeviceGuard g(h->device);
    if (int rc = materialize(h)) return rc;
    if (int rc = ensure_out(h)) return rc;
    double* dphi = h->out;
    double* dres = h->out + 3 * (size_t)h->nx * h->ny;   // the p slot, unused here
    CK(launch_macro(h, dphi, nullptr, nullptr));
    CK(launch_contact_angle(h, wall, dphi, dres));
    double res[5];
    CK(cudaMemcpyAsync(res, dres, sizeof(res), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    *theta_deg = res[0];
    if (circle) { circle[0] = res[1]; circle[1] = res[2]; circle[2] = res[3]; }
    if (npoints) *npoints = (int)res[4];
    if (res[4] < 3 || !std::isfinite(res[0])) return fail(PFLBM_EINVAL, "fewer than 3 contour points to fit");
    return read_status(h);
}

int pflbm_geometry(pflbm_t* h, uint8_t* cls, uint16_t* unknown, uint16_t* doubly, double* av)
{
    if (int rc = check_handle(h)) return rc;
    DeviceGuard g(h->device);
    size_t N = (size_t)h->nx * h->ny;
    if (cls) {
        // class bits only
        uint8_t* tmp = (uint8_t*)std::malloc((size_t)h->ny * h->pitch);
        if (!tmp) return fail(PFLBM_ENOMEM, "host allocation failed");
        cudaError_t e = cudaMemcpyAsync(tmp, h->cls, (size_t)h->ny * h->pitch, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) { std::free(tmp); return cuda_fail(e, "geometry read-back"); }
        for (int y = 0; y < h->ny; ++y)
            for (int x = 0; x < h->nx; ++x) cls[(size_t)y * h->nx + x] = tmp[(size_t)y * h->pitch + x] & CLS_MASK;
        std::free(tmp);
    }
    if (av)
        CK(cudaMemcpy2DAsync(av, h->nx * sizeof(double), h->av, h->pitch * sizeof(double), h->nx * sizeof(double),
                             h->ny, cudaMemcpyDeviceToHost, h->stream));
    if (unknown || doubly) {
        if (int rc = ensure_out(h)) return rc;
        uint16_t* du = (uint16_t*)h->out;
        uint16_t* dd = du + N;
        CK(launch_links(h, du, dd));
        if (unknown) CK(cudaMemcpyAsync(unknown, du, N * 2, cudaMemcpyDeviceToHost, h->stream));
        if (doubly) CK(cudaMemcpyAsync(doubly, dd, N * 2, cudaMemcpyDeviceToHost, h->stream));
    }
    CK(cudaStreamSynchronize(h->stream));
    return PFLBM_OK;
}

int pflbm_check(pflbm_t* h)
{
    if (int rc = check_handle(h)) return rc;
    DeviceGuard g(h->device);
    CK(cudaStreamSynchronize(h->stream));
    CK(cudaMemcpy(h->hstatus, h->dstatus, sizeof(int), cudaMemcpyDeviceToHost));
    return read_status(h);
}

int64_t pflbm_steps(const pflbm_t* h) { return h ? h->steps : -1; }

int pflbm_status(const pflbm_t* h)
{
    if (!h) return PFLBM_EINVAL;
    if (h->hstatus && (h->hstatus[0] & 4)) return PFLBM_ETIMEOUT;
    return (h->hstatus && h->hstatus[0] != 0) ? PFLBM_ENUMERIC : PFLBM_OK;
}

namespace {
// Checkpoint header. A state is only meaningful with the parameters, flags
// and geometry that produced it, so all of them are recorded and compared.
struct Blob {
    uint64_t magic;
    int32_t version, nx, ny, precision;
    int64_t steps;
    int32_t replace_phi, dgdt_mode;
    double params[10];    // beta, kappa, alpha, tau_f, tau_g, rho_l, rho_g, W, sigma, M
    double extra[4];      // nu_l, nu_g, gx, gy
    int32_t chi_case, pad;
    uint64_t geometry;    // fingerprint of the node bytes and wetting coefficients
};
constexpr uint64_t kMagic = 0x4d424c4650ULL;  // "PFLBM"
constexpr int32_t kBlobVersion = 2;

void fill_params(const Params& q, double pv[10], double ex[4])
{
    const double a[10] = {q.beta, q.kappa, q.alpha, q.tau_f, q.tau_g, q.rho_l, q.rho_g, q.W, q.sigma, q.M};
    const double b[4] = {q.nu_l, q.nu_g, q.gx, q.gy};
    std::memcpy(pv, a, sizeof(a));
    std::memcpy(ex, b, sizeof(b));
}

// Geometry fingerprint of the handle (synchronous).
int geometry_fingerprint(pflbm_t* h, uint64_t* out)
{
    unsigned long long* d = (unsigned long long*)(h->red + mass_scratch_doubles() - 16);
    CK(launch_fingerprint(h->cls, h->wet, h->precision == PFLBM_FP64, h->nx, h->ny, h->pitch, d, h->stream));
    unsigned long long v = 0;
    CK(cudaMemcpyAsync(&v, d, sizeof(v), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    *out = v;
    return PFLBM_OK;
}
}  // namespace

int pflbm_save(pflbm_t* h, void* buf, size_t* len)
{
    if (int rc = check_handle(h)) return rc;
    if (!len) return fail(PFLBM_EINVAL, "NULL len");
    Sizes s = sizes_of(h->nx, h->ny, h->precision);
    size_t need = sizeof(Blob) + s.pop + s.sprev;
    if (!buf) { *len = need; return PFLBM_OK; }
    if (*len < need) { *len = need; return fail(PFLBM_EINVAL, "buffer too small"); }
    DeviceGuard g(h->device);
    if (int rc = materialize(h)) return rc;
    Blob b{};
    b.magic = kMagic;
    b.version = kBlobVersion;
    b.nx = h->nx;
    b.ny = h->ny;
    b.precision = h->precision;
    b.steps = h->steps;
    b.replace_phi = h->replace_phi;
    b.dgdt_mode = h->prm.dgdt_mode;
    b.chi_case = h->prm.chi_case;
    fill_params(h->prm, b.params, b.extra);
    if (int rc = geometry_fingerprint(h, &b.geometry)) return rc;
    std::memcpy(buf, &b, sizeof(b));
    char* dst = (char*)buf + sizeof(Blob);
    CK(cudaMemcpyAsync(dst, h->pop[h->cur], s.pop, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(dst + s.pop, h->sprev, s.sprev, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    *len = need;
    return PFLBM_OK;
}

int pflbm_load(pflbm_t* h, const void* buf, size_t len)
{
    if (int rc = check_handle(h)) return rc;
    if (!buf || len < sizeof(Blob)) return fail(PFLBM_EINVAL, "blob too small");
    Blob b;
    std::memcpy(&b, buf, sizeof(b));
    Sizes s = sizes_of(h->nx, h->ny, h->precision);
    if (b.magic != kMagic || b.version != kBlobVersion) return fail(PFLBM_EINVAL, "not a pflbm checkpoint");
    if (b.nx != h->nx || b.ny != h->ny || b.precision != h->precision)
        return fail(PFLBM_EINVAL, "checkpoint size or precision differs from the handle");
    if (len < sizeof(Blob) + s.pop + s.sprev) return fail(PFLBM_EINVAL, "blob truncated");
    double pv[10], ex[4];
    fill_params(h->prm, pv, ex);
    if (std::memcmp(pv, b.params, sizeof(pv)) != 0 || std::memcmp(ex, b.extra, sizeof(ex)) != 0 ||
        b.dgdt_mode != h->prm.dgdt_mode || b.chi_case != h->prm.chi_case)
        return fail(PFLBM_EINVAL, "checkpoint parameters differ from the handle's");
    DeviceGuard g(h->device);
    uint64_t geo = 0;
    if (int rc = geometry_fingerprint(h, &geo)) return rc;
    if (geo != b.geometry) return fail(PFLBM_EINVAL, "checkpoint geometry or angle field differs from the handle's");
    const char* src = (const char*)buf + sizeof(Blob);
    CK(cudaMemcpyAsync(h->pop[h->cur], src, s.pop, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->sprev, src + s.pop, s.sprev, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemsetAsync(h->dstatus, 0, sizeof(int), h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (h->hstatus) h->hstatus[0] = 0;
    h->init_pending = false;
    h->steps = b.steps;
    h->replace_phi = b.replace_phi != 0;
    return PFLBM_OK;
}

}  // extern "C"
