// capi3d.cu -- the pflbm3d_* entry points of include/pflbm.h (the 3D form
// of the scheme: D3Q19 f, D3Q7 g, Sec. 2.1-2.2): argument checks, device
// memory, the handle's life cycle and the calls into the kernels of
// step3d.cu and diag3d.cu.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "pflbm3d_internal.cuh"

namespace pfk {
int set_error(int code, const char* msg);
}
using namespace pfk;
using namespace pfk3;

namespace {

size_t pop3_bytes(int prec, size_t plane)
{
    return prec == PFLBM_FP64 ? 26 * plane * 8 : 26 * plane * 4;  // g_0 plane holds its storage form
}

int fail3(int code, const std::string& m) { return set_error(code, m.c_str()); }

#define CK3(call)                                                        \
    do {                                                                 \
        cudaError_t e_ = (call);                                         \
        if (e_ != cudaSuccess) return fail3(PFLBM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

int materialize3(pflbm3d_t* h)
{
    if (!h->init_pending) return PFLBM_OK;
    CK3(launch_init(h));
    CK3(cudaMemsetAsync(h->dstatus, 0, sizeof(int), h->stream));
    if (h->hstatus) h->hstatus[0] = 0;
    h->init_pending = false;
    return PFLBM_OK;
}

// The device status word as last copied to the host (after a step or a
// check): a solve that reported NaN or |u| >= 0.3 is not stepped further.
int read_status3(const pflbm3d_t* h)
{
    if (h->hstatus && h->hstatus[0] != 0) return fail3(PFLBM_ENUMERIC, "NaN or |u| >= 0.3 detected on the device");
    return PFLBM_OK;
}

// Device buffer of `bytes` from the handle's allocator (or cudaMalloc) into *p;
// PFLBM_ENOMEM on failure.
int alloc3(pflbm3d_t* h, void** p, size_t bytes)
{
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (h->alloc_fn) {
        *p = h->alloc_fn(bytes, h->alloc_ctx);
    } else if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
    }
    if (!*p) return fail3(PFLBM_ENOMEM, h->alloc_fn ? "allocator callback returned NULL" : "cudaMalloc failed");
    h->allocs.emplace_back(*p, bytes);
    return PFLBM_OK;
}

void release3(pflbm3d_t* h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (auto& a : h->allocs) {
        if (h->free_fn)
            h->free_fn(a.first, a.second, h->alloc_ctx);
        else
            cudaFree(a.first);
    }
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    if (h->hstatus) cudaFreeHost(h->hstatus);
    delete h;
}

}  // namespace

extern "C" {

void pflbm3d_params_default(pflbm3d_params_t* p)
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

int pflbm3d_create(pflbm3d_t** out, const pflbm3d_params_t* p)
{
    if (!out || !p) return fail3(PFLBM_EINVAL, "NULL argument");
    *out = nullptr;
    if (p->nx < 3 || p->ny < 3 || p->nz < 5 || !p->solid_mask) return fail3(PFLBM_EINVAL, "need nx, ny >= 3, nz >= 5 and a mask");
    if (!(p->W > 0) || !(p->M > 0) || !(p->tau_f > 0.5) || !(p->rho_l > 0) || !(p->rho_g > 0) || !(p->sigma >= 0) ||
        (p->tau_g > 0 && !(p->tau_g > 0.5)) || !std::isfinite(p->theta_deg))
        return fail3(PFLBM_EINVAL, "invalid physical parameters");
    if (p->precision != PFLBM_FP64 && p->precision != PFLBM_FP32)
        return fail3(PFLBM_EINVAL, "3D supports PFLBM_FP64 and PFLBM_FP32");
    const int pitch = (p->nx + 63) / 64 * 64;
    const size_t plane = (size_t)p->nz * p->ny * pitch;
    if (26.0 * (double)plane >= 2147483647.0) return fail3(PFLBM_EINVAL, "lattice too large");
    if (p->nz > 65535 || (p->ny + 7) / 8 > 65535)
        return fail3(PFLBM_EINVAL, "nz must be <= 65535 and ny <= 524280 (launch grid limits)");
    const size_t pl = (size_t)p->nx * p->ny;
    for (size_t k = 0; k < pl; ++k)
        if (!p->solid_mask[k] || !p->solid_mask[pl + k] || !p->solid_mask[(p->nz - 2) * pl + k] ||
            !p->solid_mask[(p->nz - 1) * pl + k])
            return fail3(PFLBM_EBADMASK, "planes 0, 1, nz-2 and nz-1 of the solid mask must be solid");
    pflbm3d_t* h = new (std::nothrow) pflbm3d();
    if (!h) return fail3(PFLBM_ENOMEM, "host allocation failed");
    h->nx = p->nx;
    h->ny = p->ny;
    h->nz = p->nz;
    h->pitch = pitch;
    h->precision = p->precision;
    h->alloc_fn = p->alloc;
    h->free_fn = p->free;
    h->alloc_ctx = p->alloc_ctx;
    int dev = p->device;
    if (dev < 0) cudaGetDevice(&dev);
    h->device = dev;
    DeviceGuard guard(dev);
    Params& q = h->prm;
    q.sigma = p->sigma;
    q.W = p->W;
    q.M = p->M;
    q.beta = 12.0 * p->sigma / p->W;
    q.kappa = 1.5 * p->sigma * p->W;
    q.tau_f = p->tau_f;
    q.tau_g = p->tau_g > 0 ? p->tau_g : 1.0;
    q.alpha = p->M / (0.25 * (q.tau_g - 0.5));   // Eq. mobility with the D3Q7 c_s^2 = 1/4
    q.rho_l = p->rho_l;
    q.rho_g = p->rho_g;
    q.dgdt_mode = p->dgdt_mode ? 1 : 0;
    h->theta = p->theta_deg;
    if (p->stream) {
        h->stream = (cudaStream_t)p->stream;
    } else {
        cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        h->own_stream = true;
    }
    const size_t cs = p->precision == PFLBM_FP64 ? 8 : 4;
    struct B { void** ptr; size_t bytes; } bufs[] = {
        {(void**)&h->cls, plane}, {(void**)&h->solid, plane}, {(void**)&h->av, plane * 8}, {&h->wet, plane * cs},
        {&h->pop[0], pop3_bytes(p->precision, plane)}, {&h->pop[1], pop3_bytes(p->precision, plane)},
        {&h->sprev, plane * cs}, {&h->phi, plane * cs}, {(void**)&h->phi0, plane * 8}, {(void**)&h->mu0, plane * 8},
        {(void**)&h->red, (kMassBlocks + 32) * 8}, {(void**)&h->dstatus, 16}};
    for (auto& b : bufs) {
        if (int rc = alloc3(h, b.ptr, b.bytes)) {
            release3(h);
            return rc;
        }
    }
    if (cudaMallocHost((void**)&h->hstatus, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        h->hstatus = nullptr;
        release3(h);
        return fail3(PFLBM_ENOMEM, "pinned status word");
    }
    h->hstatus[0] = 0;
    cudaMemsetAsync(h->pop[0], 0, pop3_bytes(p->precision, plane), h->stream);
    cudaMemsetAsync(h->pop[1], 0, pop3_bytes(p->precision, plane), h->stream);
    cudaMemsetAsync(h->phi, 0, plane * cs, h->stream);
    cudaMemsetAsync(h->phi0, 0, plane * 8, h->stream);
    cudaMemsetAsync(h->dstatus, 0, 16, h->stream);
    cudaMemsetAsync(h->solid, 1, plane, h->stream);
    cudaMemcpy2DAsync(h->solid, pitch, p->solid_mask, p->nx, p->nx, (size_t)p->ny * p->nz, cudaMemcpyHostToDevice,
                      h->stream);
    const double coef = sqrt(2.0 * q.kappa * q.beta) * cos(h->theta * 3.14159265358979323846 / 180.0);
    launch_geometry(h, coef);
    // step path: three launches unless the fused kernel is asked for
    if (p->step_path != PFLBM3D_AUTO && p->step_path != PFLBM3D_FUSED && p->step_path != PFLBM3D_THREE_PASS) {
        release3(h);
        return fail3(PFLBM_EINVAL, "unknown step_path");
    }
    h->fused = p->step_path == PFLBM3D_FUSED;
    if (h->fused) {
        size_t sb = 0;
        int per_sm = 0, sms = 0;
        cudaError_t ea = fused_setup(p->precision, &sb, &per_sm);
        if (ea == cudaSuccess) ea = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (ea != cudaSuccess || per_sm < 1) {
            cudaGetLastError();
            release3(h);
            return fail3(PFLBM_ECUDA, "fused 3D step kernel cannot be resident");
        }
        const long long tiles = (long long)((h->nx + TX - 1) / TX) * ((h->ny + TY - 1) / TY);
        const int nzz = h->nz - 2;
        int zc = p->fused_zc;
        if (zc <= 0) {
            // about six waves of resident CTAs, 8 to 64 planes per CTA
            zc = (int)(((long long)nzz * tiles) / (6LL * sms * per_sm));
            zc = zc < 8 ? 8 : (zc > 64 ? 64 : zc);
        }
        h->fused_zc = zc > nzz ? nzz : zc;
        if (int rc = alloc3(h, (void**)&h->gflag, (size_t)tiles * h->nz)) {
            release3(h);
            return rc;
        }
        launch_ghost_flags(h);
    }
    int* cnt = h->dstatus + 1;
    cudaMemsetAsync(cnt, 0, sizeof(int), h->stream);
    launch_ghost_collect(h, cnt, nullptr);
    cudaMemcpyAsync(&h->n_ghosts, cnt, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess && h->n_ghosts > 0) {
        if (int rc = alloc3(h, (void**)&h->ghosts, (size_t)h->n_ghosts * sizeof(int))) {
            release3(h);
            return rc;
        }
        cudaMemsetAsync(cnt, 0, sizeof(int), h->stream);
        launch_ghost_collect(h, cnt, h->ghosts);
        cudaMemsetAsync(cnt, 0, sizeof(int), h->stream);
        e = cudaStreamSynchronize(h->stream);
    }
    if (e != cudaSuccess) {
        release3(h);
        return fail3(PFLBM_ECUDA, cudaGetErrorString(e));
    }
    *out = h;
    return PFLBM_OK;
}

void pflbm3d_destroy(pflbm3d_t* h)
{
    if (!h) return;
    DeviceGuard g(h->device);
    release3(h);
}

int pflbm3d_init_droplet(pflbm3d_t* h, double x0, double y0, double z0, double R)
{
    if (!h) return fail3(PFLBM_EINVAL, "NULL handle");
    DeviceGuard g(h->device);
    if (!std::isfinite(x0) || !std::isfinite(y0) || !std::isfinite(z0) || !std::isfinite(R))
        return fail3(PFLBM_EINVAL, "non-finite droplet");
    if (h->replace_phi) CK3(cudaMemsetAsync(h->phi0, 0, (size_t)h->nz * h->ny * h->pitch * 8, h->stream));
    const double reach = fabs(R) + 10.0 * h->prm.W;
    auto span = [&](double c, int n, int& lo, int& w) {
        lo = 0;
        w = n;
        if (2.0 * reach + 2.0 < n && fabs(c) < 1e8) {
            lo = (int)floor(c - reach);
            w = (int)(ceil(c + reach) - floor(c - reach)) + 1;
        }
    };
    int xlo, xw, ylo, yw;
    span(x0, h->nx, xlo, xw);
    span(y0, h->ny, ylo, yw);
    const int zlo = (int)fmin((double)h->nz, fmax(0.0, floor(z0 - reach)));
    const int zhi = (int)fmax(-1.0, fmin((double)h->nz - 1, ceil(z0 + reach)));
    if (zlo <= zhi) {
        CK3(launch_droplet(h, xlo, xw, ylo, yw, zlo, zhi - zlo + 1, x0, y0, z0, R));
    }
    h->replace_phi = false;
    h->init_pending = true;
    h->steps = 0;
    return PFLBM_OK;
}

int pflbm3d_init_phi(pflbm3d_t* h, const double* phi)
{
    if (!h || !phi) return fail3(PFLBM_EINVAL, "NULL argument");
    DeviceGuard g(h->device);
    CK3(cudaMemcpy2DAsync(h->phi0, h->pitch * 8, phi, h->nx * 8, h->nx * 8, (size_t)h->ny * h->nz,
                          cudaMemcpyHostToDevice, h->stream));
    CK3(cudaStreamSynchronize(h->stream));
    h->replace_phi = false;
    h->init_pending = true;
    h->steps = 0;
    return PFLBM_OK;
}

int pflbm3d_step(pflbm3d_t* h, int64_t n)
{
    if (!h || n < 0) return fail3(PFLBM_EINVAL, "invalid arguments");
    if (int rc = read_status3(h)) return rc;
    DeviceGuard g(h->device);
    NvtxRange range("pflbm3d_step");
    if (int rc = materialize3(h)) return rc;
    for (int64_t t = 0; t < n; ++t) {
        CK3(launch_step(h));
        h->cur ^= 1;
        h->steps += 1;
    }
    if (n > 0) {
        h->replace_phi = true;
        // refreshed without waiting; read by the next step
        CK3(cudaMemcpyAsync(h->hstatus, h->dstatus, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    }
    return PFLBM_OK;
}

int pflbm3d_get(pflbm3d_t* h, double* phi, double* u, double* p)
{
    if (!h) return fail3(PFLBM_EINVAL, "NULL handle");
    DeviceGuard g(h->device);
    if (int rc = materialize3(h)) return rc;
    const size_t N = (size_t)h->nx * h->ny * h->nz;
    if (!h->out)
        if (int rc = alloc3(h, (void**)&h->out, N * 5 * sizeof(double))) return rc;
    double *dphi = h->out, *du = h->out + N, *dp = h->out + 4 * N;
    CK3(launch_macro(h, phi ? dphi : nullptr, u ? du : nullptr, p ? dp : nullptr));
    if (phi) CK3(cudaMemcpyAsync(phi, dphi, N * 8, cudaMemcpyDeviceToHost, h->stream));
    if (u) CK3(cudaMemcpyAsync(u, du, 3 * N * 8, cudaMemcpyDeviceToHost, h->stream));
    if (p) CK3(cudaMemcpyAsync(p, dp, N * 8, cudaMemcpyDeviceToHost, h->stream));
    CK3(cudaStreamSynchronize(h->stream));
    return PFLBM_OK;
}

int pflbm3d_get_f32(pflbm3d_t* h, float* phi, float* u, float* p)
{
    if (!h) return fail3(PFLBM_EINVAL, "NULL handle");
    DeviceGuard g(h->device);
    if (int rc = materialize3(h)) return rc;
    const size_t N = (size_t)h->nx * h->ny * h->nz;
    if (!h->out_f)
        if (int rc = alloc3(h, (void**)&h->out_f, N * 5 * sizeof(float))) return rc;
    // the read-back kernel writes the float fields directly: no FP64 scratch
    float *fphi = h->out_f, *fu = h->out_f + N, *fp = h->out_f + 4 * N;
    CK3(launch_macro_f32(h, phi ? fphi : nullptr, u ? fu : nullptr, p ? fp : nullptr));
    if (phi) CK3(cudaMemcpyAsync(phi, fphi, N * 4, cudaMemcpyDeviceToHost, h->stream));
    if (u) CK3(cudaMemcpyAsync(u, fu, 3 * N * 4, cudaMemcpyDeviceToHost, h->stream));
    if (p) CK3(cudaMemcpyAsync(p, fp, N * 4, cudaMemcpyDeviceToHost, h->stream));
    CK3(cudaStreamSynchronize(h->stream));
    return PFLBM_OK;
}

int pflbm3d_mass(pflbm3d_t* h, double* out)
{
    if (!h || !out) return fail3(PFLBM_EINVAL, "NULL argument");
    DeviceGuard g(h->device);
    if (int rc = materialize3(h)) return rc;
    double* d = h->red + kMassBlocks + 4;
    CK3(launch_mass(h, d));
    CK3(cudaMemcpyAsync(out, d, 8, cudaMemcpyDeviceToHost, h->stream));
    CK3(cudaStreamSynchronize(h->stream));
    return PFLBM_OK;
}

int pflbm3d_geometry(pflbm3d_t* h, uint8_t* cls, double* av)
{
    if (!h) return fail3(PFLBM_EINVAL, "NULL handle");
    DeviceGuard g(h->device);
    if (cls) {
        CK3(cudaMemcpy2DAsync(cls, h->nx, h->cls, h->pitch, h->nx, (size_t)h->ny * h->nz, cudaMemcpyDeviceToHost,
                              h->stream));
        CK3(cudaStreamSynchronize(h->stream));
        for (size_t k = 0; k < (size_t)h->nx * h->ny * h->nz; ++k) cls[k] &= CLS_MASK;
    }
    if (av)
        CK3(cudaMemcpy2DAsync(av, h->nx * 8, h->av, h->pitch * 8, h->nx * 8, (size_t)h->ny * h->nz,
                              cudaMemcpyDeviceToHost, h->stream));
    CK3(cudaStreamSynchronize(h->stream));
    return PFLBM_OK;
}

int pflbm3d_contact_angle(pflbm3d_t* h, const pflbm3d_wall_t* wall, double* theta_deg, double* sphere, int* npoints)
{
    if (!h || !wall || !theta_deg) return fail3(PFLBM_EINVAL, "NULL argument");
    DeviceGuard g(h->device);
    if (wall->type != 0 && wall->type != 1) return fail3(PFLBM_EINVAL, "wall type must be 0 or 1");
    if (int rc = materialize3(h)) return rc;
    const size_t N = (size_t)h->nx * h->ny * h->nz;
    if (!h->out)
        if (int rc = alloc3(h, (void**)&h->out, N * 5 * sizeof(double))) return rc;
    if (!h->pts) {
        const long long cap = std::min<long long>(3LL * (long long)N, 1LL << 22);
        if (int rc = alloc3(h, (void**)&h->pts, (size_t)cap * 3 * sizeof(double))) return rc;
        h->pts_cap = (int)cap;
    }
    double* dphi = h->out;
    CK3(launch_macro(h, dphi, nullptr, nullptr));
    Wall3 w{wall->type, {wall->px, wall->py, wall->pz}, {wall->nx, wall->ny, wall->nz}, wall->r,
            wall->x_lo, wall->x_hi, wall->y_lo, wall->y_hi, wall->exclude};
    int* d_count = (int*)(h->red + kMassBlocks + 8);
    double* d_res = h->red + kMassBlocks + 16;
    CK3(launch_contact_angle3d(h->cls, dphi, h->nx, h->ny, h->nz, h->pitch, w, h->pts, h->pts_cap, d_count, d_res,
                               h->stream));
    double res[6];
    CK3(cudaMemcpyAsync(res, d_res, sizeof(res), cudaMemcpyDeviceToHost, h->stream));
    CK3(cudaStreamSynchronize(h->stream));
    *theta_deg = res[0];
    if (sphere)
        for (int i = 0; i < 4; ++i) sphere[i] = res[1 + i];
    if (npoints) *npoints = (int)res[5];
    return PFLBM_OK;
}

namespace {
constexpr uint64_t kMagic3 = 0x33444d424c46504bULL;   // checkpoint tag of the 3D state
// Checkpoint header: the parameters, flags and geometry that produced the
// state are recorded and compared on load.
struct Blob3 {
    uint64_t magic;
    int32_t version, nx, ny, nz, precision, replace_phi, dgdt_mode;
    int64_t steps;
    double params[10];    // beta, kappa, alpha, tau_f, tau_g, rho_l, rho_g, W, sigma, M
    uint64_t geometry;    // fingerprint of the node bytes and wetting coefficients
};
constexpr int32_t kBlob3Version = 2;

void params3(const Params& q, double pv[10])
{
    const double a[10] = {q.beta, q.kappa, q.alpha, q.tau_f, q.tau_g, q.rho_l, q.rho_g, q.W, q.sigma, q.M};
    std::memcpy(pv, a, sizeof(a));
}

int fingerprint3(pflbm3d_t* h, uint64_t* out)
{
    unsigned long long* d = (unsigned long long*)(h->red + kMassBlocks + 2);
    CK3(launch_fingerprint(h->cls, h->wet, h->precision == PFLBM_FP64, h->nx, (long long)h->ny * h->nz, h->pitch, d,
                           h->stream));
    unsigned long long v = 0;
    CK3(cudaMemcpyAsync(&v, d, sizeof(v), cudaMemcpyDeviceToHost, h->stream));
    CK3(cudaStreamSynchronize(h->stream));
    *out = v;
    return PFLBM_OK;
}
size_t sprev3_bytes(const pflbm3d_t* h)
{
    return (size_t)h->nz * h->ny * h->pitch * (h->precision == PFLBM_FP64 ? 8 : 4);
}
}  // namespace

int pflbm3d_save(pflbm3d_t* h, void* buf, size_t* len)
{
    if (!h || !len) return fail3(PFLBM_EINVAL, "NULL argument");
    const size_t plane = (size_t)h->nz * h->ny * h->pitch;
    const size_t pop = pop3_bytes(h->precision, plane), sp = sprev3_bytes(h);
    const size_t need = sizeof(Blob3) + pop + sp;
    if (!buf) { *len = need; return PFLBM_OK; }
    if (*len < need) { *len = need; return fail3(PFLBM_EINVAL, "buffer too small"); }
    DeviceGuard g(h->device);
    if (int rc = materialize3(h)) return rc;
    Blob3 b{};
    b.magic = kMagic3;
    b.version = kBlob3Version;
    b.dgdt_mode = h->prm.dgdt_mode;
    if (int rc = fingerprint3(h, &b.geometry)) return rc;
    b.nx = h->nx;
    b.ny = h->ny;
    b.nz = h->nz;
    b.precision = h->precision;
    b.replace_phi = h->replace_phi;
    b.steps = h->steps;
    params3(h->prm, b.params);
    std::memcpy(buf, &b, sizeof(b));
    char* dst = (char*)buf + sizeof(Blob3);
    CK3(cudaMemcpyAsync(dst, h->pop[h->cur], pop, cudaMemcpyDeviceToHost, h->stream));
    CK3(cudaMemcpyAsync(dst + pop, h->sprev, sp, cudaMemcpyDeviceToHost, h->stream));
    CK3(cudaStreamSynchronize(h->stream));
    *len = need;
    return PFLBM_OK;
}

int pflbm3d_load(pflbm3d_t* h, const void* buf, size_t len)
{
    if (!h || !buf || len < sizeof(Blob3)) return fail3(PFLBM_EINVAL, "blob too small");
    Blob3 b;
    std::memcpy(&b, buf, sizeof(b));
    if (b.magic != kMagic3 || b.version != kBlob3Version) return fail3(PFLBM_EINVAL, "not a pflbm3d checkpoint");
    if (b.nx != h->nx || b.ny != h->ny || b.nz != h->nz || b.precision != h->precision)
        return fail3(PFLBM_EINVAL, "checkpoint size or precision differs from the handle");
    const size_t plane = (size_t)h->nz * h->ny * h->pitch;
    const size_t pop = pop3_bytes(h->precision, plane), sp = sprev3_bytes(h);
    if (len < sizeof(Blob3) + pop + sp) return fail3(PFLBM_EINVAL, "blob truncated");
    double pv[10];
    params3(h->prm, pv);
    if (std::memcmp(pv, b.params, sizeof(pv)) != 0 || b.dgdt_mode != h->prm.dgdt_mode)
        return fail3(PFLBM_EINVAL, "checkpoint parameters differ from the handle's");
    DeviceGuard g(h->device);
    uint64_t geo = 0;
    if (int rc = fingerprint3(h, &geo)) return rc;
    if (geo != b.geometry) return fail3(PFLBM_EINVAL, "checkpoint geometry differs from the handle's");
    const char* src = (const char*)buf + sizeof(Blob3);
    CK3(cudaMemcpyAsync(h->pop[h->cur], src, pop, cudaMemcpyHostToDevice, h->stream));
    CK3(cudaMemcpyAsync(h->sprev, src + pop, sp, cudaMemcpyHostToDevice, h->stream));
    CK3(cudaMemsetAsync(h->dstatus, 0, sizeof(int), h->stream));
    CK3(cudaStreamSynchronize(h->stream));
    if (h->hstatus) h->hstatus[0] = 0;
    h->init_pending = false;
    h->steps = b.steps;
    h->replace_phi = b.replace_phi != 0;
    return PFLBM_OK;
}

int64_t pflbm3d_steps(const pflbm3d_t* h) { return h ? h->steps : -1; }

int pflbm3d_check(pflbm3d_t* h)
{
    if (!h) return fail3(PFLBM_EINVAL, "NULL handle");
    DeviceGuard g(h->device);
    CK3(cudaStreamSynchronize(h->stream));
    int st = 0;
    CK3(cudaMemcpy(&st, h->dstatus, sizeof(int), cudaMemcpyDeviceToHost));
    if (h->hstatus) h->hstatus[0] = st;
    return st ? fail3(PFLBM_ENUMERIC, "NaN or |u| >= 0.3 detected on the device") : PFLBM_OK;
}

}  // extern "C"
