// geometry.cu -- node classification and the effective surface area a_v
// (Sec. 2.2.2 and Sec. 2.2.3), once per handle. Integer work; a_v is exact:
// with epsilon in {0, 1}, grad(epsilon) = n / 12 with the integer vector
// n = sum_i w36_i c_i epsilon(x + c_i), w36 = 36 w_i = (4 axes, 1 diagonals),
// so a_v = sqrt(n.n) / 12 is one correctly rounded sqrt and one division.
#include "pflbm_internal.cuh"

namespace pfk {
namespace {

__device__ inline int wrapx(int x, int nx) { return x < 0 ? x + nx : (x >= nx ? x - nx : x); }

// Pass 1: fluid / boundary / (tentatively) interior from the solid mask.
__global__ void k_classify_1(const uint8_t* __restrict__ solid, uint8_t* __restrict__ cls,
                             int nx, int ny, int pitch)
{
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= nx || y >= ny) return;
    size_t k = (size_t)y * pitch + x;
    uint8_t c;
    if (!solid[k]) {
        c = CLS_FLUID;
    } else {
        bool touches = false;
        for (int i = 1; i < 9; ++i) {
            int yy = y + cy(i);
            if (yy < 0 || yy >= ny) continue;
            if (!solid[(size_t)yy * pitch + wrapx(x + cx(i), nx)]) touches = true;
        }
        c = touches ? CLS_BOUNDARY : CLS_INTERIOR;
    }
    cls[k] = c;
}

// Pass 2: interior nodes next to a zeta = 1 node become ghosts.
__global__ void k_classify_2(uint8_t* __restrict__ cls, int nx, int ny, int pitch)
{
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= nx || y >= ny) return;
    size_t k = (size_t)y * pitch + x;
    if (cls[k] != CLS_INTERIOR) return;
    for (int i = 1; i < 9; ++i) {
        int yy = y + cy(i);
        if (yy < 0 || yy >= ny) continue;
        uint8_t c = cls[(size_t)yy * pitch + wrapx(x + cx(i), nx)];
        // pass 1 wrote only FLUID / BOUNDARY / INTERIOR; a concurrent
        // INTERIOR -> GHOST update of a neighbour does not change zeta.
        if ((c & CLS_MASK) <= CLS_BOUNDARY) {
            cls[k] = CLS_GHOST;
            return;
        }
    }
}

// Pass 3: a_v, the flag bits, and zero a_v elsewhere.
__global__ void k_classify_3(uint8_t* __restrict__ cls, double* __restrict__ av, int nx,
                             int ny, int pitch, int chi_case)
{
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= nx || y >= ny) return;
    size_t k = (size_t)y * pitch + x;
    uint8_t c = cls[k] & CLS_MASK;
    double a = 0.0;
    uint8_t flags = 0;
    if (c <= CLS_BOUNDARY) {
        int n_x = 0, n_y = 0;
        for (int i = 1; i < 9; ++i) {
            int yy = y + cy(i);  // in range: rows 0 and ny-1 are never zeta = 1
            uint8_t cn = cls[(size_t)yy * pitch + wrapx(x + cx(i), nx)] & CLS_MASK;
            int w36 = (i <= 4) ? 4 : 1;
            int eps = (cn == CLS_FLUID) ? 1 : 0;
            n_x += w36 * cx(i) * eps;
            n_y += w36 * cy(i) * eps;
            if (cn > CLS_BOUNDARY) flags |= F_LINK;
            if (cn == CLS_GHOST) flags |= F_NEARGHOST;
        }
        if (n_x != 0 || n_y != 0) {
            a = sqrt((double)(n_x * n_x + n_y * n_y)) / 12.0;
            flags |= F_WET;
        }
    }
    if (c == CLS_GHOST && chi_case != 2) {
        // Appendix A cases 1 and 3: a ghost node of a flat wall has exactly one
        // zeta = 1 node straight above or below it; other ghosts keep the mean
        bool up = y + 1 < ny && (cls[(size_t)(y + 1) * pitch + x] & CLS_MASK) <= CLS_BOUNDARY;
        bool dn = y >= 1 && (cls[(size_t)(y - 1) * pitch + x] & CLS_MASK) <= CLS_BOUNDARY;
        if (up != dn) flags = up ? F_GHOST_UP : F_GHOST_DOWN;
    }
    av[k] = a;
    // pass 3 reads only the class bits of neighbours, so writing the flag
    // bits of this node concurrently is safe
    cls[k] = c | flags;
}

// Wetting coefficient per zeta = 1 node: factor a_v sqrt(2 kappa beta)
// cos(theta), factor = 1 (the paper's method), 0 (Appendix A case 1) or 2
// (case 3). Robin ghost nodes (cases 1 and 3) hold instead the coefficient
// c = -/+ sqrt(2 beta / kappa) cos(theta) of chi = c (phi - phi^2), with the
// angle of their mirror node.
template <typename C>
__global__ void k_wet(const uint8_t* __restrict__ cls, const double* __restrict__ av,
                      const float* __restrict__ theta, C* __restrict__ wet, double root,
                      double theta_uniform, int nx, int ny, int pitch, double factor, double chi_c)
{
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= nx || y >= ny) return;
    size_t k = (size_t)y * pitch + x;
    const uint8_t code = cls[k];
    if ((code & CLS_MASK) == CLS_GHOST && (code & (F_GHOST_UP | F_GHOST_DOWN))) {
        size_t b = (code & F_GHOST_UP) ? k + pitch : k - pitch;
        double thb = theta ? (double)theta[b] : theta_uniform;
        wet[k] = (C)(chi_c * cos(thb * 3.14159265358979323846 / 180.0));
        return;
    }
    const double a = av[k] * factor;
    if (a == 0.0) { wet[k] = (C)0; return; }
    double th = theta ? (double)theta[k] : theta_uniform;
    // Eq. chemical_potencial2: the wall term is a_v sqrt(2 kappa beta) cos(theta) (phi - phi^2)
    wet[k] = (C)(a * root * cos(th * 3.14159265358979323846 / 180.0));
}

__global__ void k_links(const uint8_t* __restrict__ cls, uint16_t* __restrict__ unknown,
                        uint16_t* __restrict__ doubly, int nx, int ny, int pitch)
{
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= nx || y >= ny) return;
    size_t k = (size_t)y * pitch + x;
    uint16_t un = 0, db = 0;
    if (zeta_of(cls[k])) {
        for (int i = 1; i < 9; ++i) {
            uint8_t src = cls[(size_t)(y - cy(i)) * pitch + wrapx(x - cx(i), nx)];
            uint8_t dst = cls[(size_t)(y + cy(i)) * pitch + wrapx(x + cx(i), nx)];
            if (!zeta_of(src)) {
                un |= (uint16_t)(1u << i);
                if (!zeta_of(dst)) db |= (uint16_t)(1u << i);
            }
        }
    }
    size_t o = (size_t)y * nx + x;  // dense output
    if (unknown) unknown[o] = un;
    if (doubly) doubly[o] = db;
}

// Per step tile: 1 when every node within two nodes of the tile (x periodic)
// exists and is a fluid node, so the step can skip the class tile, the
// bounce-back checks, the ghost fill and the wetting term there. Needs
// nx >= 2 TX so that one wrap covers the tile's halo.
__global__ void k_tile_flags(const uint8_t* __restrict__ cls, uint8_t* __restrict__ tiles, int nx, int ny,
                             int pitch, int ntx, int nty)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntx * nty) return;
    int bx = t % ntx, by = t / ntx;
    int x0 = bx * TX, y0 = by * TY;
    uint8_t ok = (nx >= 2 * TX) ? 1 : 0;
    for (int y = y0 - 2; ok && y < y0 + TY + 2; ++y) {
        if (y < 0 || y >= ny) { ok = 0; break; }
        for (int x = x0 - 2; x < x0 + TX + 2; ++x) {
            int xx = x < 0 ? x + nx : (x >= nx ? x - nx : x);
            if ((cls[(size_t)y * pitch + xx] & CLS_MASK) != CLS_FLUID) { ok = 0; break; }
        }
    }
    tiles[t] = ok;
}

dim3 grid2d(int nx, int ny, dim3 b) { return dim3((nx + b.x - 1) / b.x, (ny + b.y - 1) / b.y); }

// SplitMix64 finaliser (Steele, Lea and Flood, OOPSLA 2014): a bijective
// mixing of 64 bits.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Fingerprint of a geometry: the sum (mod 2^64) over the nodes of a hash of
// (node index, node byte, bit pattern of the wetting coefficient). Integer
// addition is order-free, so the result does not depend on the launch.
template <typename C>
__global__ void k_fingerprint(const uint8_t* __restrict__ cls, const C* __restrict__ wet, int nx, long long rows,
                              int pitch, unsigned long long* out)
{
    unsigned long long acc = 0;
    const long long n = rows * nx;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / nx, x = i - r * nx;
        const size_t k = (size_t)r * pitch + x;
        unsigned long long wb;
        if constexpr (sizeof(C) == 8) wb = (unsigned long long)__double_as_longlong((double)wet[k]);
        else wb = (unsigned long long)(unsigned)__float_as_int((float)wet[k]);
        acc += mix64(mix64(((unsigned long long)i << 8) | cls[k]) ^ wb);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

// Per TXT x TYT tile of the staged step (tile column sx, block b): bit 0 when
// every node within two of the tile's nodes lies in the lattice and is a
// fluid node (no class reads, no bounce-back checks, no ghosts: the fluid
// path), bit 1 when a node of the tile is a ghost or a zeta = 1 node next to
// a ghost (the phi tile then needs a ring of two and the ghost values).
template <int TXT, int TYT>
__global__ void k_staged_flags(const uint8_t* __restrict__ cls, uint8_t* __restrict__ flags, int nx, int ny, int pitch,
                               int nsx, int nby)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nsx * nby) return;
    const int sx = t % nsx, b = t / nsx;
    const int x0 = sx * TXT, y0 = b * TYT, nreal = min(TXT, nx - x0);
    auto at = [&](int x, int y) {
        int xx = x % nx;
        if (xx < 0) xx += nx;
        return cls[(size_t)y * pitch + xx];
    };
    bool fluid = true;
    for (int y = y0 - 2; fluid && y < y0 + TYT + 2; ++y) {
        if (y < 0 || y >= ny) { fluid = false; break; }
        for (int x = x0 - 2; x < x0 + nreal + 2; ++x)
            if ((at(x, y) & CLS_MASK) != CLS_FLUID) { fluid = false; break; }
    }
    bool halo2 = false;
    for (int y = y0; y < min(y0 + TYT, ny); ++y)
        for (int x = x0; x < x0 + nreal; ++x) {
            const uint8_t c = at(x, y);
            if ((zeta_of(c) && (c & F_NEARGHOST)) || (c & CLS_MASK) == CLS_GHOST) halo2 = true;
        }
    flags[t] = (fluid ? 1 : 0) | (halo2 ? 2 : 0);
}

}  // namespace

// Node words of the two-node step: the node byte in the low byte and, in the
// high byte, bit j - 1 = zeta(x + c_j) for j = 1..8 (x periodic; rows outside
// the lattice are not zeta = 1 nodes). With it a node's bounce-back sources
// (Sec. 2.2.2) and a ghost node's zeta-weighted neighbour mean need no class
// tile. Padding columns hold CLS_OUT.
__global__ void k_node_words(const uint8_t* __restrict__ cls, uint16_t* __restrict__ words, int nx, int ny, int pitch)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= pitch || y >= ny) return;
    if (x >= nx) {
        words[(size_t)y * pitch + x] = CLS_OUT;
        return;
    }
    unsigned m = 0;
    for (int j = 1; j < 9; ++j) {
        const int yy = y + cy(j), xx = ((x + cx(j)) % nx + nx) % nx;
        if (yy >= 0 && yy < ny && zeta_of(cls[(size_t)yy * pitch + xx])) m |= 1u << (j - 1);
    }
    words[(size_t)y * pitch + x] = (uint16_t)(cls[(size_t)y * pitch + x] | (m << 8));
}

// Flags of the two-node step's 64 x 8 tiles: bit 0 both 32 x 8 halves are
// all-fluid tiles (a right half past the lattice counts as fluid); bit 1 the
// tile needs phi two nodes out (a zeta = 1 node next to a ghost, or a ghost
// node, among its nodes, a column past nx - 1 standing for its periodic
// image); bit 2 the tile has a zeta = 1 node (x < nx): a tile without one
// stores nothing, and the step skips it.
__global__ void k_tile2_flags(const uint8_t* __restrict__ cls, const uint8_t* __restrict__ tiles,
                              uint8_t* __restrict__ tiles2, int nx, int ny, int pitch)
{
    const int ntx = (nx + 31) / 32, ntx2 = (nx + 63) / 64, nty = (ny + 7) / 8;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntx2 * nty) return;
    const int bx = t % ntx2, by = t / ntx2;
    uint8_t f = (tiles[by * ntx + 2 * bx] != 0 && (2 * bx + 1 >= ntx || tiles[by * ntx + 2 * bx + 1] != 0)) ? 1 : 0;
    for (int y = by * 8; y < by * 8 + 8 && y < ny; ++y)
        for (int x = bx * 64; x < bx * 64 + 64; ++x) {
            const uint8_t c = cls[(size_t)y * pitch + x % nx];
            if ((zeta_of(c) && (c & F_NEARGHOST)) || (c & CLS_MASK) == CLS_GHOST) f |= 2;
            if (x < nx && zeta_of(c)) f |= 4;
        }
    tiles2[t] = f;
}

size_t node_words_bytes(int nx, int ny) { return (size_t)ny * ((nx + 63) / 64 * 64) * sizeof(uint16_t); }
size_t tile2_flags_bytes(int nx, int ny) { return (size_t)((nx + 63) / 64) * ((ny + 7) / 8); }

cudaError_t launch_node_words(pflbm_t* h)
{
    dim3 b(64, 4), g((h->pitch + 63) / 64, (h->ny + 3) / 4);
    k_node_words<<<g, b, 0, h->stream>>>(h->cls, h->nword, h->nx, h->ny, h->pitch);
    const int n = ((h->nx + 63) / 64) * ((h->ny + 7) / 8);
    k_tile2_flags<<<(n + 127) / 128, 128, 0, h->stream>>>(h->cls, h->tiles, h->tiles2, h->nx, h->ny, h->pitch);
    return cudaGetLastError();
}

size_t staged_flags_bytes(int nx, int ny)
{
    return (size_t)((nx + 31) / 32) * ((ny + 7) / 8) + (size_t)((nx + 63) / 64) * ((ny + 3) / 4);
}

cudaError_t launch_staged_flags(pflbm_t* h)
{
    const int n0 = ((h->nx + 31) / 32) * ((h->ny + 7) / 8), n1 = ((h->nx + 63) / 64) * ((h->ny + 3) / 4);
    k_staged_flags<32, 8><<<(n0 + 127) / 128, 128, 0, h->stream>>>(h->cls, h->sflags, h->nx, h->ny, h->pitch,
                                                                  (h->nx + 31) / 32, (h->ny + 7) / 8);
    k_staged_flags<64, 4><<<(n1 + 127) / 128, 128, 0, h->stream>>>(h->cls, h->sflags + n0, h->nx, h->ny, h->pitch,
                                                                  (h->nx + 63) / 64, (h->ny + 3) / 4);
    return cudaGetLastError();
}

cudaError_t launch_fingerprint(const uint8_t* cls, const void* wet, bool wet_fp64, int nx, long long rows, int pitch,
                               unsigned long long* d_out, cudaStream_t stream)
{
    cudaError_t e = cudaMemsetAsync(d_out, 0, sizeof(unsigned long long), stream);
    if (e != cudaSuccess) return e;
    long long n = rows * nx, blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    if (wet_fp64)
        k_fingerprint<double><<<(int)blocks, 256, 0, stream>>>(cls, (const double*)wet, nx, rows, pitch, d_out);
    else
        k_fingerprint<float><<<(int)blocks, 256, 0, stream>>>(cls, (const float*)wet, nx, rows, pitch, d_out);
    return cudaGetLastError();
}

cudaError_t launch_tile_flags(pflbm_t* h)
{
    int ntx = tiles_x(h->nx), nty = tiles_y(h->ny), n = ntx * nty;
    k_tile_flags<<<(n + 127) / 128, 128, 0, h->stream>>>(h->cls, h->tiles, h->nx, h->ny, h->pitch, ntx, nty);
    return cudaGetLastError();
}

cudaError_t launch_classify(pflbm_t* h)
{
    dim3 b(32, 8), g = grid2d(h->nx, h->ny, b);
    k_classify_1<<<g, b, 0, h->stream>>>(h->solid, h->cls, h->nx, h->ny, h->pitch);
    k_classify_2<<<g, b, 0, h->stream>>>(h->cls, h->nx, h->ny, h->pitch);
    k_classify_3<<<g, b, 0, h->stream>>>(h->cls, h->av, h->nx, h->ny, h->pitch, h->prm.chi_case);
    return cudaGetLastError();
}

cudaError_t launch_wet(pflbm_t* h)
{
    dim3 b(32, 8), g = grid2d(h->nx, h->ny, b);
    double root = sqrt(2.0 * h->prm.kappa * h->prm.beta);
    const int cc = h->prm.chi_case;
    double factor = cc == 1 ? 0.0 : (cc == 3 ? 2.0 : 1.0);
    double chi_c = (cc == 1 ? -1.0 : 1.0) * sqrt(2.0 * h->prm.beta / h->prm.kappa);
    if (h->precision == PFLBM_FP64)
        k_wet<double><<<g, b, 0, h->stream>>>(h->cls, h->av, h->theta, (double*)h->wet, root,
                                              h->theta_uniform, h->nx, h->ny, h->pitch, factor, chi_c);
    else
        k_wet<float><<<g, b, 0, h->stream>>>(h->cls, h->av, h->theta, (float*)h->wet, root,
                                             h->theta_uniform, h->nx, h->ny, h->pitch, factor, chi_c);
    return cudaGetLastError();
}

cudaError_t launch_links(pflbm_t* h, uint16_t* unknown, uint16_t* doubly)
{
    dim3 b(32, 8), g = grid2d(h->nx, h->ny, b);
    k_links<<<g, b, 0, h->stream>>>(h->cls, unknown, doubly, h->nx, h->ny, h->pitch);
    return cudaGetLastError();
}

}  // namespace pfk
