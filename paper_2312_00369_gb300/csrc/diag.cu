// diag.cu -- FP64 diagnostics: the phi mass and the contact-angle fit.
// Both are reductions in FP64 with warp shuffles and a fixed block order
// (the mass is bit-reproducible run to run).
#include "storage.cuh"

namespace pfk {
namespace {

constexpr int RB = 256;         // reduction block
constexpr int MASS_BLOCKS = 1216;  // 8 per SM on 152 SMs

__device__ __forceinline__ int wrap1(int x, int nx) { return x < 0 ? x + nx : (x >= nx ? x - nx : x); }

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the block; the result is valid in thread 0.
template <int NT>
__device__ double block_sum(double v, double* sh)
{
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        r = (lane < NT / 32) ? sh[lane] : 0.0;
        r = warp_sum(r);
    }
    return r;
}

// Pulled g_I at node (x, y), same rule as the step, as a double.
template <int PREC, int I>
__device__ __forceinline__ double pulled_g(const Planes<PREC>& P, const uint8_t* __restrict__ cls, int x, int y,
                                           int nx, int pitch, size_t plane)
{
    using T = Store<PREC>;
    constexpr int X = cx(I), Y = cy(I), O = opp(I);
    size_t src = (size_t)(y - Y) * pitch + wrap1(x - X, nx);
    if (zeta_of(cls[src])) return (double)T::template ld<I>(P.g[I * plane + src]);
    size_t dst = (size_t)(y + Y) * pitch + wrap1(x + X, nx);
    if (zeta_of(cls[dst])) return (double)T::template ld<O>(P.g[O * plane + dst]);
    return (double)T::template ld<O>(P.g[O * plane + (size_t)y * pitch + x]);
}

template <int PREC>
__global__ void __launch_bounds__(RB) k_mass_partial(const uint8_t* __restrict__ cls, Planes<PREC> P, int nx, int ny,
                                                     int pitch, size_t plane, double* __restrict__ partial)
{
    __shared__ double sh[RB / 32];
    double acc = 0.0;
    const long long N = (long long)nx * ny;
    for (long long t = (long long)blockIdx.x * RB + threadIdx.x; t < N; t += (long long)gridDim.x * RB) {
        int y = (int)(t / nx), x = (int)(t - (long long)y * nx);
        if (!zeta_of(cls[(size_t)y * pitch + x])) continue;
        double v0 = Store<PREC>::g0_double(P.g0[(size_t)y * pitch + x]);
        double v1 = pulled_g<PREC, 1>(P, cls, x, y, nx, pitch, plane);
        double v2 = pulled_g<PREC, 2>(P, cls, x, y, nx, pitch, plane);
        double v3 = pulled_g<PREC, 3>(P, cls, x, y, nx, pitch, plane);
        double v4 = pulled_g<PREC, 4>(P, cls, x, y, nx, pitch, plane);
        double v5 = pulled_g<PREC, 5>(P, cls, x, y, nx, pitch, plane);
        double v6 = pulled_g<PREC, 6>(P, cls, x, y, nx, pitch, plane);
        double v7 = pulled_g<PREC, 7>(P, cls, x, y, nx, pitch, plane);
        double v8 = pulled_g<PREC, 8>(P, cls, x, y, nx, pitch, plane);
        acc += ((v0 + v1) + (v2 + v3)) + ((v4 + v5) + (v6 + v7)) + v8;
    }
    double r = block_sum<RB>(acc, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = r;
}

__global__ void __launch_bounds__(RB) k_sum_partials(const double* __restrict__ partial, int n,
                                                     double* __restrict__ out)
{
    __shared__ double sh[RB / 32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += RB) acc += partial[i];
    double r = block_sum<RB>(acc, sh);
    if (threadIdx.x == 0) *out = r;
}

// ---------------------------------------------------------------------------
// Contact angle: phi = 1/2 crossings between fluid neighbours, then a circle
// fit (algebraic fit on mean-centred points, Gauss-Newton on the geometric
// distance), then the angle against the wall, all in FP64.
// ---------------------------------------------------------------------------
struct Wall {
    int type;
    double px, py, nx, ny, r, x_lo, x_hi, exclude;
};

__device__ __forceinline__ double wall_distance(const Wall& w, double x, double y)
{
    if (w.type == 0) return (x - w.px) * w.nx + (y - w.py) * w.ny;
    double dx = x - w.px, dy = y - w.py;
    return sqrt(dx * dx + dy * dy) - w.r;
}

__global__ void k_crossings(const uint8_t* __restrict__ cls, const double* __restrict__ phi, int nx, int ny,
                            int pitch, Wall w, double* __restrict__ pts, int cap, int* __restrict__ count)
{
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= nx || y >= ny) return;
    if ((cls[(size_t)y * pitch + x] & CLS_MASK) != CLS_FLUID) return;
    double a = phi[(size_t)y * nx + x];
    for (int dir = 0; dir < 2; ++dir) {
        int xx = x + (dir == 0), yy = y + (dir == 1);
        if (xx >= nx || yy >= ny) continue;
        if ((cls[(size_t)yy * pitch + xx] & CLS_MASK) != CLS_FLUID) continue;
        double b = phi[(size_t)yy * nx + xx];
        if ((a >= 0.5) == (b >= 0.5)) continue;
        double t = (0.5 - a) / (b - a);
        double qx = x + (dir == 0 ? t : 0.0), qy = y + (dir == 1 ? t : 0.0);
        if (qx < w.x_lo || qx >= w.x_hi) continue;
        if (wall_distance(w, qx, qy) <= w.exclude) continue;
        int k = atomicAdd(count, 1);
        if (k < cap) {
            pts[2 * k] = qx;
            pts[2 * k + 1] = qy;
        }
    }
}

__device__ bool solve3(double A[3][3], double b[3], double z[3])
{
    for (int c = 0; c < 3; ++c) {
        int piv = c;
        for (int r = c + 1; r < 3; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (A[piv][c] == 0.0) return false;
        if (piv != c) {
            for (int k = 0; k < 3; ++k) { double t = A[c][k]; A[c][k] = A[piv][k]; A[piv][k] = t; }
            double t = b[c]; b[c] = b[piv]; b[piv] = t;
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
    return true;
}

constexpr int FB = 512;

// out = {theta_deg, a, b, R, n}
__global__ void __launch_bounds__(FB) k_fit(const double* __restrict__ pts, const int* __restrict__ count, int cap,
                                            Wall w, double* __restrict__ out)
{
    __shared__ double sh[FB / 32];
    __shared__ double bc[4];
    __shared__ int flag;
    int n = *count;
    if (n > cap) n = cap;
    if (n < 3) {
        if (threadIdx.x == 0) { out[0] = nan(""); out[1] = out[2] = out[3] = 0.0; out[4] = n; }
        return;
    }
    // mean
    double sx = 0, sy = 0;
    for (int k = threadIdx.x; k < n; k += FB) { sx += pts[2 * k]; sy += pts[2 * k + 1]; }
    sx = block_sum<FB>(sx, sh);
    sy = block_sum<FB>(sy, sh);
    if (threadIdx.x == 0) { bc[0] = sx / n; bc[1] = sy / n; }
    __syncthreads();
    const double mx = bc[0], my = bc[1];
    // algebraic fit: normal equations of min sum (u^2 + v^2 + D u + E v + F)^2
    double m[9] = {0};
    for (int k = threadIdx.x; k < n; k += FB) {
        double u = pts[2 * k] - mx, v = pts[2 * k + 1] - my, rhs = -(u * u + v * v);
        m[0] += u * u; m[1] += u * v; m[2] += u; m[3] += v * v; m[4] += v; m[5] += 1.0;
        m[6] += u * rhs; m[7] += v * rhs; m[8] += rhs;
    }
    double tot[9];
    for (int j = 0; j < 9; ++j) tot[j] = block_sum<FB>(m[j], sh);
    if (threadIdx.x == 0) {
        double A[3][3] = {{tot[0], tot[1], tot[2]}, {tot[1], tot[3], tot[4]}, {tot[2], tot[4], tot[5]}};
        double b[3] = {tot[6], tot[7], tot[8]}, z[3];
        flag = 0;
        if (solve3(A, b, z)) {
            double a0 = -z[0] / 2.0, b0 = -z[1] / 2.0, R2 = a0 * a0 + b0 * b0 - z[2];
            if (R2 > 0) { bc[0] = a0; bc[1] = b0; bc[2] = sqrt(R2); flag = 1; }
        }
    }
    __syncthreads();
    if (!flag) {
        if (threadIdx.x == 0) { out[0] = nan(""); out[4] = 0; }
        return;
    }
    for (int it = 0; it < 50; ++it) {
        const double a0 = bc[0], b0 = bc[1], R = bc[2];
        double q[9] = {0};
        for (int k = threadIdx.x; k < n; k += FB) {
            double u = pts[2 * k] - mx - a0, v = pts[2 * k + 1] - my - b0;
            double d = sqrt(u * u + v * v);
            if (d == 0.0) continue;
            double J0 = -u / d, J1 = -v / d, J2 = -1.0, r = d - R;
            q[0] += J0 * J0; q[1] += J0 * J1; q[2] += J0 * J2; q[3] += J1 * J1; q[4] += J1 * J2; q[5] += J2 * J2;
            q[6] -= J0 * r; q[7] -= J1 * r; q[8] -= J2 * r;
        }
        for (int j = 0; j < 9; ++j) tot[j] = block_sum<FB>(q[j], sh);
        if (threadIdx.x == 0) {
            double A[3][3] = {{tot[0], tot[1], tot[2]}, {tot[1], tot[3], tot[4]}, {tot[2], tot[4], tot[5]}};
            double b[3] = {tot[6], tot[7], tot[8]}, dz[3];
            flag = 0;
            if (solve3(A, b, dz)) {
                bc[0] = a0 + dz[0]; bc[1] = b0 + dz[1]; bc[2] = R + dz[2];
                flag = (fabs(dz[0]) + fabs(dz[1]) + fabs(dz[2]) < 1e-13 * (1.0 + fabs(R))) ? 0 : 1;
            }
        }
        __syncthreads();
        if (!flag) break;
    }
    if (threadIdx.x == 0) {
        double a0 = bc[0] + mx, b0 = bc[1] + my, R = bc[2], ct;
        if (w.type == 0) {
            ct = -((a0 - w.px) * w.nx + (b0 - w.py) * w.ny) / R;
        } else {
            double dx = a0 - w.px, dy = b0 - w.py;
            ct = (R * R + w.r * w.r - (dx * dx + dy * dy)) / (2.0 * R * w.r);
        }
        ct = fmin(1.0, fmax(-1.0, ct));
        out[0] = acos(ct) * (180.0 / 3.14159265358979323846);
        out[1] = a0; out[2] = b0; out[3] = R; out[4] = n;
    }
}

}  // namespace

template <int PREC>
void mass_prec(pflbm_t* h, size_t plane)
{
    k_mass_partial<PREC><<<MASS_BLOCKS, RB, 0, h->stream>>>(h->cls, Planes<PREC>::make(h->pop[h->cur], plane), h->nx,
                                                            h->ny, h->pitch, plane, h->red);
}

cudaError_t launch_mass(pflbm_t* h, double* d_out)
{
    size_t plane = (size_t)h->ny * h->pitch;
    switch (h->precision) {
        case PFLBM_FP64: mass_prec<PFLBM_FP64>(h, plane); break;
        case PFLBM_FP32: mass_prec<PFLBM_FP32>(h, plane); break;
        case PFLBM_BF16: mass_prec<PFLBM_BF16>(h, plane); break;
        default: mass_prec<PFLBM_FP16>(h, plane); break;
    }
    k_sum_partials<<<1, RB, 0, h->stream>>>(h->red, MASS_BLOCKS, d_out);
    return cudaGetLastError();
}

size_t mass_scratch_doubles() { return MASS_BLOCKS + 16; }

cudaError_t launch_contact_angle(pflbm_t* h, const pflbm_wall_t* wall, const double* d_phi, double* d_result)
{
    Wall w{wall->type, wall->px, wall->py, wall->nx, wall->ny, wall->r, wall->x_lo, wall->x_hi, wall->exclude};
    int* d_count = (int*)(h->red + MASS_BLOCKS + 8);
    cudaMemsetAsync(d_count, 0, sizeof(int), h->stream);
    dim3 b(32, 8), g((h->nx + 31) / 32, (h->ny + 7) / 8);
    k_crossings<<<g, b, 0, h->stream>>>(h->cls, d_phi, h->nx, h->ny, h->pitch, w, h->pts, h->pts_cap, d_count);
    k_fit<<<1, FB, 0, h->stream>>>(h->pts, d_count, h->pts_cap, w, d_result);
    return cudaGetLastError();
}

}  // namespace pfk
