// pflbm3d_internal.cuh -- the 3D handle (pflbm3d_t of include/pflbm.h) and
// the launch functions that step3d.cu (kernels) provides to capi3d.cu (the
// pflbm3d_* entry points). Not part of the ABI.
#pragma once

#include <utility>
#include <vector>

#include "pflbm_internal.cuh"

struct pflbm3d {
    int nx = 0, ny = 0, nz = 0, pitch = 0, precision = PFLBM_FP32, device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    pfk::Params prm{};
    double theta = 90.0;
    uint8_t* cls = nullptr;
    uint8_t* solid = nullptr;
    double* av = nullptr;
    void* wet = nullptr;
    void* pop[2] = {nullptr, nullptr};
    void* sprev = nullptr;
    void* phi = nullptr;
    double* phi0 = nullptr;
    double* mu0 = nullptr;
    double* red = nullptr;
    double* out = nullptr;
    float* out_f = nullptr;     // FP32 read-back scratch (5 dense fields), on first use
    int* dstatus = nullptr;
    int* hstatus = nullptr;     // pinned host mirror of dstatus[0], refreshed after each pflbm3d_step
    double* pts = nullptr;      // contact-angle crossings (3 doubles each)
    int pts_cap = 0;
    int* ghosts = nullptr;      // indices of the ghost nodes
    int n_ghosts = 0;
    bool fused = true;          // one-launch step (k3_fused) or three launches
    uint8_t* gflag = nullptr;   // [nz][tiles]: a ghost in the tile's 34 x 10 window
    int fused_zc = 0;           // planes per CTA of the fused step
    int cur = 0;
    bool replace_phi = true, init_pending = false;
    int64_t steps = 0;
    // optional device allocator (both NULL: cudaMalloc / cudaFree)
    void* (*alloc_fn)(size_t, void*) = nullptr;
    void (*free_fn)(void*, size_t, void*) = nullptr;
    void* alloc_ctx = nullptr;
    std::vector<std::pair<void*, size_t>> allocs;   // every device buffer, freed at destroy
};

namespace pfk3 {

constexpr int kMassBlocks = 1216;   // FP64 mass partials (8 per SM on 152 SMs)

// one time step (fused or three launches, as h->fused says)
cudaError_t launch_step(pflbm3d_t* h);
// phi, u, p of the current state into dense device arrays [nz][ny][nx] (any may be NULL)
cudaError_t launch_macro(pflbm3d_t* h, double* phi, double* u, double* p);
// the same fields rounded to float (round to nearest)
cudaError_t launch_macro_f32(pflbm3d_t* h, float* phi, float* u, float* p);
// initial populations from h->phi0 (ghost fill, mu, f = 0, g = g^eq)
cudaError_t launch_init(pflbm3d_t* h);
// sum of the pulled g over zeta = 1 nodes into *d_out (FP64, fixed order)
cudaError_t launch_mass(pflbm3d_t* h, double* d_out);
// classes, a_v and the wetting coefficient a_v * wet_coef from h->solid
cudaError_t launch_geometry(pflbm3d_t* h, double wet_coef);
// ghost nodes: count into *count (device), and their indices into list if not NULL
cudaError_t launch_ghost_collect(pflbm3d_t* h, int* count, int* list);
// per tile and plane: a ghost in the tile's 34 x 10 window (h->gflag)
cudaError_t launch_ghost_flags(pflbm3d_t* h);
// Eq. initialphi on the bounding box [xlo, xlo + xw) x [ylo, ylo + yw) x [zlo, zlo + zn)
cudaError_t launch_droplet(pflbm3d_t* h, int xlo, int xw, int ylo, int yw, int zlo, int zn, double x0, double y0,
                           double z0, double R);
// shared-memory attribute and resident CTAs per SM of the fused step kernel
cudaError_t fused_setup(int precision, size_t* smem_bytes, int* ctas_per_sm);

}  // namespace pfk3
