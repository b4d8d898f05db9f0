// diag3d.cu -- FP64 contact-angle fit of a three-dimensional droplet: the
// phi = 1/2 crossings between fluid neighbours (linear interpolation along
// x, y and z), a sphere fit (algebraic start, then Gauss-Newton on the
// geometric distance) in one block with warp-shuffle reductions, and the
// angle against a plane wall or a solid sphere (the 3D counterpart of the
// circle fit on the walls of Secs. 3.1-3.3).
#include "pflbm_internal.cuh"

namespace pfk {
namespace {

constexpr int FB3 = 512;

__device__ __forceinline__ double warp_sum3(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the block in a fixed order; the result is valid in every thread.
__device__ double block_sum3(double v, double* sh, double* bcast)
{
    v = warp_sum3(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    if (wid == 0) {
        double r = lane < FB3 / 32 ? sh[lane] : 0.0;
        r = warp_sum3(r);
        if (lane == 0) *bcast = r;
    }
    __syncthreads();
    return *bcast;
}

__device__ __forceinline__ double wall_distance3(const Wall3& w, double x, double y, double z)
{
    if (w.type == 0) return (x - w.p[0]) * w.n[0] + (y - w.p[1]) * w.n[1] + (z - w.p[2]) * w.n[2];
    const double dx = x - w.p[0], dy = y - w.p[1], dz = z - w.p[2];
    return sqrt(dx * dx + dy * dy + dz * dz) - w.r;
}

__global__ void k3_crossings(const uint8_t* __restrict__ cls, const double* __restrict__ phi, int nx, int ny, int nz,
                             int pitch, Wall3 w, double* __restrict__ pts, int cap, int* __restrict__ count)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y, z = blockIdx.z;
    if (x >= nx || y >= ny) return;
    if ((cls[((size_t)z * ny + y) * pitch + x] & CLS_MASK) != CLS_FLUID) return;
    const double a = phi[((size_t)z * ny + y) * nx + x];
    for (int d = 0; d < 3; ++d) {
        const int xx = x + (d == 0), yy = y + (d == 1), zz = z + (d == 2);
        if (xx >= nx || yy >= ny || zz >= nz) continue;
        if ((cls[((size_t)zz * ny + yy) * pitch + xx] & CLS_MASK) != CLS_FLUID) continue;
        const double b = phi[((size_t)zz * ny + yy) * nx + xx];
        if ((a >= 0.5) == (b >= 0.5)) continue;
        const double t = (0.5 - a) / (b - a);
        const double qx = x + (d == 0 ? t : 0.0), qy = y + (d == 1 ? t : 0.0), qz = z + (d == 2 ? t : 0.0);
        if (qx < w.x_lo || qx >= w.x_hi || qy < w.y_lo || qy >= w.y_hi) continue;
        if (wall_distance3(w, qx, qy, qz) <= w.exclude) continue;
        const int k = atomicAdd(count, 1);
        if (k < cap) {
            pts[3 * k] = qx;
            pts[3 * k + 1] = qy;
            pts[3 * k + 2] = qz;
        }
    }
}

// Gaussian elimination with partial pivoting, 4 x 4.
__device__ bool solve4(double A[4][4], double b[4], double z[4])
{
    for (int c = 0; c < 4; ++c) {
        int piv = c;
        for (int r = c + 1; r < 4; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (A[piv][c] == 0.0) return false;
        if (piv != c) {
            for (int k = 0; k < 4; ++k) { const double t = A[c][k]; A[c][k] = A[piv][k]; A[piv][k] = t; }
            const double t = b[c]; b[c] = b[piv]; b[piv] = t;
        }
        for (int r = c + 1; r < 4; ++r) {
            const double m = A[r][c] / A[c][c];
            for (int k = c; k < 4; ++k) A[r][k] -= m * A[c][k];
            b[r] -= m * b[c];
        }
    }
    for (int r = 3; r >= 0; --r) {
        double acc = b[r];
        for (int k = r + 1; k < 4; ++k) acc -= A[r][k] * z[k];
        z[r] = acc / A[r][r];
    }
    return true;
}

// Symmetric 4 x 4 from its upper triangle (10 sums) and a right-hand side.
__device__ void unpack4(const double t[14], double A[4][4], double b[4])
{
    int q = 0;
    for (int i = 0; i < 4; ++i)
        for (int j = i; j < 4; ++j) A[i][j] = A[j][i] = t[q++];
    for (int i = 0; i < 4; ++i) b[i] = t[10 + i];
}

// out = {theta_deg, cx, cy, cz, R, n}
__global__ void __launch_bounds__(FB3) k3_fit(const double* __restrict__ pts, const int* __restrict__ count, int cap,
                                              Wall3 w, double* __restrict__ out)
{
    __shared__ double sh[FB3 / 32];
    __shared__ double bcast;
    __shared__ double sol[4];
    __shared__ int go;
    int n = *count;
    if (n > cap) n = cap;
    if (n < 4) {
        if (threadIdx.x == 0) {
            out[0] = nan("");
            out[1] = out[2] = out[3] = out[4] = 0.0;
            out[5] = n;
        }
        return;
    }
    double m[3] = {0, 0, 0};
    for (int k = threadIdx.x; k < n; k += FB3)
        for (int d = 0; d < 3; ++d) m[d] += pts[3 * k + d];
    for (int d = 0; d < 3; ++d) m[d] = block_sum3(m[d], sh, &bcast) / n;
    // algebraic fit on centred points: min sum (|r|^2 + D.r + F)^2
    double t[14];
    for (int j = 0; j < 14; ++j) t[j] = 0.0;
    for (int k = threadIdx.x; k < n; k += FB3) {
        const double r[4] = {pts[3 * k] - m[0], pts[3 * k + 1] - m[1], pts[3 * k + 2] - m[2], 1.0};
        const double rhs = -(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        int q = 0;
        for (int i = 0; i < 4; ++i)
            for (int j = i; j < 4; ++j) t[q++] += r[i] * r[j];
        for (int i = 0; i < 4; ++i) t[10 + i] += r[i] * rhs;
    }
    for (int j = 0; j < 14; ++j) t[j] = block_sum3(t[j], sh, &bcast);
    if (threadIdx.x == 0) {
        double A[4][4], b[4], z[4];
        unpack4(t, A, b);
        go = 0;
        if (solve4(A, b, z)) {
            const double c0 = -z[0] / 2.0, c1 = -z[1] / 2.0, c2 = -z[2] / 2.0;
            const double R2 = c0 * c0 + c1 * c1 + c2 * c2 - z[3];
            if (R2 > 0) {
                sol[0] = c0; sol[1] = c1; sol[2] = c2; sol[3] = sqrt(R2);
                go = 1;
            }
        }
    }
    __syncthreads();
    if (!go) {
        if (threadIdx.x == 0) { out[0] = nan(""); out[5] = 0; }
        return;
    }
    for (int it = 0; it < 50; ++it) {
        const double c0 = sol[0], c1 = sol[1], c2 = sol[2], R = sol[3];
        for (int j = 0; j < 14; ++j) t[j] = 0.0;
        for (int k = threadIdx.x; k < n; k += FB3) {
            const double u0 = pts[3 * k] - m[0] - c0, u1 = pts[3 * k + 1] - m[1] - c1, u2 = pts[3 * k + 2] - m[2] - c2;
            const double dd = sqrt(u0 * u0 + u1 * u1 + u2 * u2);
            if (dd == 0.0) continue;
            const double J[4] = {-u0 / dd, -u1 / dd, -u2 / dd, -1.0}, r = dd - R;
            int q = 0;
            for (int i = 0; i < 4; ++i)
                for (int j = i; j < 4; ++j) t[q++] += J[i] * J[j];
            for (int i = 0; i < 4; ++i) t[10 + i] -= J[i] * r;
        }
        for (int j = 0; j < 14; ++j) t[j] = block_sum3(t[j], sh, &bcast);
        if (threadIdx.x == 0) {
            double A[4][4], b[4], dz[4];
            unpack4(t, A, b);
            go = 0;
            if (solve4(A, b, dz)) {
                sol[0] = c0 + dz[0]; sol[1] = c1 + dz[1]; sol[2] = c2 + dz[2]; sol[3] = R + dz[3];
                go = (fabs(dz[0]) + fabs(dz[1]) + fabs(dz[2]) + fabs(dz[3]) < 1e-13 * (1.0 + fabs(R))) ? 0 : 1;
            }
        }
        __syncthreads();
        if (!go) break;
    }
    if (threadIdx.x == 0) {
        const double c0 = sol[0] + m[0], c1 = sol[1] + m[1], c2 = sol[2] + m[2], R = sol[3];
        double ct;
        if (w.type == 0) {
            ct = -((c0 - w.p[0]) * w.n[0] + (c1 - w.p[1]) * w.n[1] + (c2 - w.p[2]) * w.n[2]) / R;
        } else {
            const double d0 = c0 - w.p[0], d1 = c1 - w.p[1], d2 = c2 - w.p[2];
            ct = (R * R + w.r * w.r - (d0 * d0 + d1 * d1 + d2 * d2)) / (2.0 * R * w.r);
        }
        ct = fmin(1.0, fmax(-1.0, ct));
        out[0] = acos(ct) * (180.0 / 3.14159265358979323846);
        out[1] = c0; out[2] = c1; out[3] = c2; out[4] = R; out[5] = n;
    }
}

}  // namespace

cudaError_t launch_contact_angle3d(const uint8_t* cls, const double* d_phi, int nx, int ny, int nz, int pitch,
                                   const Wall3& w, double* pts, int cap, int* d_count, double* d_out,
                                   cudaStream_t stream)
{
    cudaError_t e = cudaMemsetAsync(d_count, 0, sizeof(int), stream);
    if (e != cudaSuccess) return e;
    dim3 b(32, 8), g((nx + 31) / 32, (ny + 7) / 8, nz);
    k3_crossings<<<g, b, 0, stream>>>(cls, d_phi, nx, ny, nz, pitch, w, pts, cap, d_count);
    k3_fit<<<1, FB3, 0, stream>>>(pts, d_count, cap, w, d_out);
    return cudaGetLastError();
}

}  // namespace pfk
