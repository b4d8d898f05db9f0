// pflbm_internal.cuh -- shared definitions of the CUDA library (not part of
// the ABI): lattice constants, the handle layout, kernel entry points.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <vector>

#include <cstddef>
#include <cstdint>

#include "../../include/pflbm.h"

namespace pfk {

// ---------------------------------------------------------------------------
// D2Q9 in the library's order: rest, the four axes counter-clockwise from +x,
// then the four diagonals counter-clockwise from (+1,+1). Weights 4/9, 1/9,
// 1/36 and c_s^2 = 1/3 (Sec. 2.1.2).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int cx(int i) { return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0); }
__host__ __device__ constexpr int cy(int i) { return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0); }
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 5 + 2) % 4) + 5); }

template <typename C> __host__ __device__ constexpr C wgt(int i) {
    return i == 0 ? C(4) / C(9) : (i <= 4 ? C(1) / C(9) : C(1) / C(36));
}

// Node byte: bits 0-1 class, bit 2 "a_v != 0" (read the wetting coefficient),
// bit 3 "zeta = 1 with a zeta = 0 neighbour" (bounce-back links present),
// bit 4 "ghost node in the 8-neighbourhood" (stencil reaches a ghost value).
// For ghost nodes bits 2-3 mean instead "Robin ghost (Appendix A cases 1
// and 3) whose flat-wall mirror node is straight above / below".
enum : uint8_t {
    CLS_FLUID = 0, CLS_BOUNDARY = 1, CLS_GHOST = 2, CLS_INTERIOR = 3,
    CLS_MASK = 3, F_WET = 4, F_LINK = 8, F_NEARGHOST = 16,
    F_GHOST_UP = 4, F_GHOST_DOWN = 8,
    CLS_OUT = 0xFF  // outside the lattice in y (tile halos only)
};
__host__ __device__ inline bool zeta_of(uint8_t c) { return c != CLS_OUT && (c & CLS_MASK) <= CLS_BOUNDARY; }

// Multiply-add with one rounding. The library is compiled without implicit
// contraction (-fmad=false): every fused multiply-add in it is written as one
// of these, so a formula rounds the same way in every kernel that inlines it
// (single-lattice, batched, fused and three-pass steps agree bit for bit).
__device__ __forceinline__ float fmadd(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmadd(double a, double b, double c) { return fma(a, b, c); }

// c . v for a lattice velocity c with components in {-1, 0, 1}, without
// multiplications (x * 0 cannot be folded under IEEE rules).
template <int X, int Y, typename C>
__device__ __forceinline__ C cdot(C vx, C vy)
{
    static_assert(X >= -1 && X <= 1 && Y >= -1 && Y <= 1 && (X || Y), "lattice velocity");
    if constexpr (X == 0) return Y > 0 ? vy : -vy;
    else if constexpr (Y == 0) return X > 0 ? vx : -vx;
    else if constexpr (X > 0) return Y > 0 ? vx + vy : vx - vy;
    else return Y > 0 ? vy - vx : -(vx + vy);
}
template <int X, int Y, int Z, typename C>
__device__ __forceinline__ C cdot(C vx, C vy, C vz)
{
    static_assert(X >= -1 && X <= 1 && Y >= -1 && Y <= 1 && Z >= -1 && Z <= 1 && (X || Y || Z), "lattice velocity");
    static_assert(!(X && Y && Z), "D3Q19 velocity");
    if constexpr (Z == 0) return cdot<X, Y>(vx, vy);
    else if constexpr (X == 0 && Y == 0) return Z > 0 ? vz : -vz;
    else if constexpr (X == 0) return cdot<Y, Z>(vy, vz);
    else return cdot<X, Z>(vx, vz);
}

// Makes `dev` the current device for the life of the guard and restores the
// caller's device on return: every entry point that touches the device
// takes one, so a caller that switched devices after creating a handle still
// runs that handle's work on the handle's device.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
    DeviceGuard(const DeviceGuard&) = delete;
    DeviceGuard& operator=(const DeviceGuard&) = delete;
};

// NVTX range around an entry point's device work (visible in Nsight tools;
// a no-op without one attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Tile of the fused step: TX x TY nodes per CTA, one node per thread.
constexpr int TX = 32;
constexpr int TY = 8;

// Wall of the 3D contact-angle fit (pflbm3d_wall_t on the device).
struct Wall3 {
    int type;             // 0 plane through p with unit normal n into the fluid; 1 solid sphere (p, r)
    double p[3], n[3], r;
    double x_lo, x_hi, y_lo, y_hi, exclude;
};
cudaError_t launch_contact_angle3d(const uint8_t* cls, const double* d_phi, int nx, int ny, int nz, int pitch,
                                   const Wall3& w, double* pts, int cap, int* d_count, double* d_out,
                                   cudaStream_t stream);

struct Params {           // derived parameters (Sec. 2.1-2.2), in FP64
    double beta, kappa, alpha, tau_f, tau_g, rho_l, rho_g, W, sigma, M;
    double nu_l, nu_g;    // both > 0: variable viscosity
    double gx, gy;        // body acceleration
    int dgdt_mode;        // 0 backward difference of G, 1 omitted
    int chi_case;         // Appendix A, Table 2: 1, 2 (the paper's method) or 3
};

struct TmaSet;            // tensor maps of the staged step (step_core.cuh)

}  // namespace pfk

// The handle.
struct pflbm {
    int nx = 0, ny = 0, pitch = 0;
    int precision = PFLBM_FP32;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    pfk::Params prm{};
    double theta_uniform = 90.0;
    // allocator
    void* (*alloc_fn)(size_t, void*) = nullptr;
    void (*free_fn)(void*, size_t, void*) = nullptr;
    void* alloc_ctx = nullptr;
    // device buffers (sizes: N = ny*pitch nodes)
    uint8_t* cls = nullptr;       // node byte [N]
    uint8_t* tiles = nullptr;     // per step tile: 1 = all nodes within 2 are fluid
    uint16_t* nword = nullptr;    // two-node step (FP32, 16-bit): node byte | zeta-neighbour bits << 8 [N]
    uint8_t* tiles2 = nullptr;    // two-node step: per 64 x 8 tile, bit 0 all fluid, bit 1 halo of two,
                                  // bit 2 has a zeta = 1 node
    uint8_t* solid = nullptr;     // user mask [N]
    float* theta = nullptr;       // angle field [N] (degrees)
    void* wet = nullptr;          // a_v sqrt(2 kappa beta) cos(theta) [N] (FP64 or FP32)
    double* av = nullptr;         // a_v [N]
    void* pop[2] = {nullptr, nullptr};  // f then g, each [9][ny][pitch], ping-pong
    void* sprev = nullptr;        // u.grad(phi) history [N]
    double* phi0 = nullptr;       // initial-field staging / ghost-filled phi [N]
    double* mu0 = nullptr;        // initial chemical potential [N]
    double* red = nullptr;        // reduction scratch
    double* pts = nullptr;        // contact-angle points (2 * pts_cap)
    int pts_cap = 0;
    double* out = nullptr;        // read-back scratch (4 dense [ny][nx] doubles)
    size_t out_bytes = 0;
    float* out_f = nullptr;       // FP32 read-back scratch (4 dense [ny][nx] floats), on first use
    int* dstatus = nullptr;       // device status word
    int* hstatus = nullptr;       // pinned host mirror
    int cur = 0;                  // which pop buffer holds the current state
    bool replace_phi = true;
    bool init_pending = false;    // phi0 set, populations not yet built
    int64_t steps = 0;
    size_t bytes_allocated = 0;
    cudaEvent_t status_ev = nullptr;
    // staged step (FP32 and 16-bit): tensor maps [shape][copy] in device memory
    pfk::TmaSet* tma = nullptr;
    uint8_t* sflags = nullptr;    // staged step: per-tile flags of both shapes
    int step_shape = -1;          // -1: global-load step kernel; 0: 32 x 8; 1: 64 x 4 staged;
                                  // -2: global loads, two nodes per thread (packed FP32x2)
    int step_chunk = 16;          // staged step: tiles per work item (blocks a CTA marches)
};

namespace pfk {

size_t elem_size(int precision);
size_t pop_bytes(int ny, int pitch, int precision);   // one of f or g, one copy

// geometry.cu
cudaError_t launch_classify(pflbm_t* h);
cudaError_t launch_wet(pflbm_t* h);
cudaError_t launch_links(pflbm_t* h, uint16_t* unknown, uint16_t* doubly);
cudaError_t launch_tile_flags(pflbm_t* h);
// tile flags of the staged step for both tile shapes (h->sflags: the 32 x 8
// tiles, then the 64 x 4 tiles, tile column fastest)
size_t staged_flags_bytes(int nx, int ny);
cudaError_t launch_staged_flags(pflbm_t* h);
// Order-free 64-bit fingerprint of the node bytes and wetting coefficients of
// a [rows][pitch] lattice (first nx columns) into *d_out: checkpoints record
// it so that a state is only loaded into a handle of the same geometry.
cudaError_t launch_fingerprint(const uint8_t* cls, const void* wet, bool wet_fp64, int nx, long long rows, int pitch,
                               unsigned long long* d_out, cudaStream_t stream);
__host__ __device__ inline int tiles_x(int nx) { return (nx + TX - 1) / TX; }
__host__ __device__ inline int tiles_y(int ny) { return (ny + TY - 1) / TY; }

// step.cu
cudaError_t launch_init_phi_droplet(pflbm_t* h, double x0, double y0, double R, int replace);
cudaError_t launch_init_populations(pflbm_t* h);
cudaError_t launch_step(pflbm_t* h);
// step2.cu: two x-adjacent nodes per thread in packed FP32x2 (FP32, 16-bit)
cudaError_t launch_step2(pflbm_t* h);
size_t node_words_bytes(int nx, int ny);
size_t tile2_flags_bytes(int nx, int ny);
cudaError_t launch_node_words(pflbm_t* h);   // nword and tiles2 from cls and tiles
// two-node kernel over up to step2_class_capacity() lattices of one size
// (nx, ny) and one viscosity mode: descs holds their step descriptors
// (count x step_args_bytes, host memory, copied into the launch)
int step2_class_capacity(int precision);
cudaError_t launch_step2_class(int precision, int vv, const unsigned char* descs, int count, int nx, int ny,
                               cudaStream_t stream);
cudaError_t launch_macro(pflbm_t* h, double* phi, double* u, double* p);
cudaError_t launch_macro_f32(pflbm_t* h, float* phi, float* u, float* p);   // rounded to nearest
size_t step_args_bytes(int precision);
void write_step_args(pflbm_t* h, int flip, void* dst);   // flip: in/out swapped
cudaError_t launch_step_batch(int precision, const void* d_args, const int2* d_work, int n_work, int group,
                              int grid, cudaStream_t stream);
int batch_max_ctas_per_sm(int precision);

// step_tma.cu: the staged step (TMA ring, tile shapes 0: 32 x 8, 1: 64 x 4)
constexpr int kStagedShapes = 2;
struct TmaSet;
size_t tma_sets_bytes();   // kStagedShapes x 2 copies of TmaSet, then 2 copies of PfMaps
bool encode_tma_sets(const pflbm_t* h, TmaSet* host);      // false: staged step unavailable
cudaError_t launch_step_staged(pflbm_t* h, int shape, int blocks_per_item, int ctas_per_sm);
cudaError_t launch_step_staged_batch(int precision, const void* d_args, const int4* d_work, int n_work, int grid,
                                     cudaStream_t stream);
int staged_batch_ctas_per_sm(int precision);
// index-checked build: out-of-range accesses counted in step.cu / step_tma.cu
unsigned bounds_violations_step();
unsigned bounds_violations_tma();
unsigned bounds_violations_step2();

// diag.cu
cudaError_t launch_mass(pflbm_t* h, double* d_out);
cudaError_t launch_contact_angle(pflbm_t* h, const pflbm_wall_t* wall, const double* d_phi,
                                 double* d_result /* theta, a, b, R, n */);

}  // namespace pfk
