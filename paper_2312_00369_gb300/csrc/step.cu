// step.cu -- initial state, the fused time step and the macroscopic read-back.
//
// The stored values are POST-COLLISION populations f*_i(x), g*_i(x) at the
// node that produced them (pull scheme; storage formats in storage.cuh). A
// step at node x first pulls its post-streaming populations,
//     f_i(x) = f*_i(x - c_i)          if zeta(x - c_i) = 1   (streaming)
//            = f*_{i'}(x + c_i)       else if zeta(x + c_i) = 1
//            = f*_{i'}(x)             otherwise,
// which is the modified bounce-back of Sec. 2.2.2 (unknown f_i(x_b) takes the
// post-streaming f_{i'}(x_b); if that is unknown too, the node's own
// post-collision f*_{i'}). Then it computes phi = sum g_i (Eq.
// order-parameter) on a shared-memory tile with a one- or two-node halo,
// fills ghost nodes with the zeta-weighted neighbour mean (Sec. 2.2.2), takes
// the isotropic gradient and Laplacian (Eqs. gradient, Laplace), the chemical
// potential with the wetting term (Eq. chemical_potencial2), rho, the force
// F = mu grad(phi), u and p (Sec. 2.1.2), collides f (Eqs. BGK-NS, feq_i, Siu,
// GGi) and g (Eqs. BGK, H_i, F_i with (1/2) dG/dt as a backward difference)
// and stores f*, g* and the new u.grad(phi) history.
//
// g_0 carries phi (it is O(1) while every other population is O(alpha mu)),
// so rounding it on every store is what limits a 32-bit state: outside FP64
// it is a 32-bit fixed-point number advanced by integer addition of the
// collision increment g*_0 - g_0 = (g_0^eq - g_0)/tau_g + (3/2 G_0(t) -
// 1/2 G_0(t-1)), where g_0^eq - g_0 = sum_{i!=0} g_i - (1 - w_0) alpha mu holds
// no O(1) term.
#include "step_core.cuh"

#ifndef PFLBM_BATCH_MINB
#define PFLBM_BATCH_MINB 5   // resident 256-thread CTAs per SM asked of k_step_batch (FP32, 16-bit)
#endif
#ifndef PFLBM_PREFETCH_F_WALL
#define PFLBM_PREFETCH_F_WALL 0   // tiles with walls: pull f with g, before the phi-tile barriers
#endif
#ifndef PFLBM_PREFETCH_F
#define PFLBM_PREFETCH_F 0   // fluid tiles: pull f before the phi-tile barrier
#endif
#ifndef PFLBM_STEP_MINB
#define PFLBM_STEP_MINB 6    // resident 256-thread CTAs per SM asked of k_step (FP32, 16-bit)
#endif
#ifndef PFLBM_L2_AHEAD
// k_step: prefetch into L2 the rows of the tile this many CTAs later in
// launch order (0: off). With 6 resident CTAs on each of 152 SMs, 228 is a
// quarter of a wave: about 1.5 us before that CTA starts, short enough that
// the lines are still in L2 when it reads them (measured optimum; at a whole
// wave and beyond the lines are evicted first and the step slows down).
#define PFLBM_L2_AHEAD 228
#endif

namespace pfk {
namespace {

// Prologue of a tile whose nodes within two of it are all fluid: no class
// tile, no bounce-back checks, no ghosts, phi on a one-node ring.
template <int PREC, bool WRAP>
__device__ __forceinline__ void tile_prologue_fluid(const StepArgs<PREC>& a,
                                                    typename Store<PREC>::C (*s_phi)[TX + 4], int x0, int y0,
                                                    typename Store<PREC>::C gown[9],
                                                    typename Store<PREC>::G0T& raw0,
                                                    typename Store<PREC>::C fown[9])
{
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * TX + tx;
    const int nx = a.nx, pitch = a.pitch, plane = a.plane;
    {
        const int gx = WRAP ? wrap1(x0 + tx, nx) : x0 + tx, gy = y0 + ty;
        pull_g<PREC, false, WRAP>(gown, raw0, a.in, nullptr, 0, 0, gx, gy, nx, pitch, plane);
        // the f pulls do not depend on phi: issue them before the barrier
        if (PFLBM_PREFETCH_F) pull_f<PREC, false, WRAP>(fown, a.in.f, nullptr, 0, 0, gx, gy, nx, pitch, plane);
        s_phi[ty + 2][tx + 2] = phi_of<PREC>(gown);
    }
    // ring: top row, bottom row (TX + 2 each), left and right columns (TY each)
    constexpr int RT = TX + 2, NR = 2 * (TX + 2) + 2 * TY;
    if (tid < NR) {
        int py, px;
        if (tid < RT) { py = 1; px = 1 + tid; }
        else if (tid < 2 * RT) { py = TY + 2; px = 1 + tid - RT; }
        else if (tid < 2 * RT + TY) { py = 2 + tid - 2 * RT; px = 1; }
        else { py = 2 + tid - 2 * RT - TY; px = TX + 2; }
        const int gy = y0 - 2 + py, gx = WRAP ? wrap1(x0 - 2 + px, nx) : x0 - 2 + px;
        s_phi[py][px] = pulled_phi<PREC, false, WRAP>(a.in, nullptr, 0, 0, gx, gy, nx, pitch, plane);
    }
    __syncthreads();
}

// phi on the ring of width H around the tile (one position per thread).
template <int PREC, int H, bool WRAP>
__device__ __forceinline__ void ring_phi(const StepArgs<PREC>& a, const uint8_t (*s_cls)[TX + 6],
                                         typename Store<PREC>::C (*s_phi)[TX + 4], int x0, int y0, int tid,
                                         bool tiny)
{
    using C = typename Store<PREC>::C;
    constexpr int RW = TX + 2 * H, NTOP = H * RW, NSIDE = H * TY;
    static_assert(2 * NTOP + 2 * NSIDE <= TX * TY, "one ring position per thread");
    if (tid >= 2 * NTOP + 2 * NSIDE) return;
    int py, px;
    if (tid < NTOP) {
        py = 2 - H + tid / RW;
        px = 2 - H + tid % RW;
    } else if (tid < 2 * NTOP) {
        const int t = tid - NTOP;
        py = TY + 2 + t / RW;
        px = 2 - H + t % RW;
    } else if (tid < 2 * NTOP + NSIDE) {
        const int t = tid - 2 * NTOP;
        py = 2 + t / H;
        px = 2 - H + t % H;
    } else {
        const int t = tid - 2 * NTOP - NSIDE;
        py = 2 + t / H;
        px = TX + 2 + t % H;
    }
    const int sy = py + 1, sx = px + 1;
    C ph = C(0);
    const uint8_t c = s_cls[sy][sx];
    if (zeta_of(c)) {
        const int gy = y0 - 2 + py, xr = x0 - 2 + px;
        const int gx = !WRAP ? xr : (tiny ? wrapn(xr, a.nx) : wrap1(xr, a.nx));
        if (has_link(c))
            ph = pulled_phi<PREC, true, WRAP>(a.in, s_cls, sy, sx, gx, gy, a.nx, a.pitch, a.plane);
        else
            ph = pulled_phi<PREC, false, WRAP>(a.in, s_cls, sy, sx, gx, gy, a.nx, a.pitch, a.plane);
    }
    s_phi[py][px] = ph;
}

// General prologue: class tile (halo 3) and phi tile with ghost values. A
// tile needs phi two nodes out only when a ghost node lies next to one of its
// nodes (the ghost average reaches one node further); otherwise one ring.
// Returns the own node's pulled g (and raw g_0) when it is a zeta = 1 node.
template <int PREC, bool WRAP>
__device__ __forceinline__ void tile_prologue(const StepArgs<PREC>& a, uint8_t (*s_cls)[TX + 6],
                                              typename Store<PREC>::C (*s_phi)[TX + 4], int x0, int y0,
                                              typename Store<PREC>::C gown[9], typename Store<PREC>::G0T& raw0,
                                              typename Store<PREC>::C fown[9])
{
    using C = typename Store<PREC>::C;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * TX + tx;
    const int nx = a.nx, ny = a.ny, pitch = a.pitch;

    // one conditional wrap covers the tile and its halo unless nx is tiny
    const bool tiny = nx < TX + 8;
    auto wx = [&](int x) { return !WRAP ? x : (tiny ? wrapn(x, nx) : wrap1(x, nx)); };
    for (int p = tid; p < (TY + 6) * (TX + 6); p += TX * TY) {
        int py = p / (TX + 6), px = p - py * (TX + 6);
        int gy = y0 - 3 + py, gx = wx(x0 - 3 + px);
        s_cls[py][px] = (gy < 0 || gy >= ny) ? (uint8_t)CLS_OUT : PFLBM_LD(a.cls, gy * pitch + gx, a.plane);
    }
    __syncthreads();
    const uint8_t own = s_cls[ty + 3][tx + 3];
    // halo 2 when a node of the tile reads a ghost value: a zeta = 1 node next
    // to a ghost, or a ghost node itself (its value is part of the read-back)
    const bool near_ghost = (y0 + ty < ny) && own != CLS_OUT &&
                            ((zeta_of(own) && (own & F_NEARGHOST)) || (own & CLS_MASK) == CLS_GHOST);
    const int halo = __syncthreads_or(near_ghost) ? 2 : 1;

    // own node (a tile that runs past x = nx - 1 holds wrapped nodes there:
    // they are computed like halo nodes but not collided)
    {
        int gx = wx(x0 + tx), gy = y0 + ty;
        C ph = C(0);
        if (gy < ny && zeta_of(own)) {
            if (has_link(own)) {
                pull_g<PREC, true, WRAP>(gown, raw0, a.in, s_cls, ty + 3, tx + 3, gx, gy, nx, pitch, a.plane);
                if (PFLBM_PREFETCH_F_WALL)
                    pull_f<PREC, true, WRAP>(fown, a.in.f, s_cls, ty + 3, tx + 3, gx, gy, nx, pitch, a.plane);
            } else {
                pull_g<PREC, false, WRAP>(gown, raw0, a.in, s_cls, ty + 3, tx + 3, gx, gy, nx, pitch, a.plane);
                if (PFLBM_PREFETCH_F_WALL)
                    pull_f<PREC, false, WRAP>(fown, a.in.f, s_cls, ty + 3, tx + 3, gx, gy, nx, pitch, a.plane);
            }
            ph = phi_of<PREC>(gown);
        }
        s_phi[ty + 2][tx + 2] = ph;
    }
    // halo ring of width 1 or 2: top rows, bottom rows, left and right columns
    if (halo == 1)
        ring_phi<PREC, 1, WRAP>(a, s_cls, s_phi, x0, y0, tid, tiny);
    else
        ring_phi<PREC, 2, WRAP>(a, s_cls, s_phi, x0, y0, tid, tiny);
    __syncthreads();
    if (halo == 1) return;

    // ghost nodes within one node of the tile: zeta-weighted 3x3 mean, or
    // the Robin value of Appendix A cases 1 and 3 on flat walls
    fill_ghosts<C, TX, TY, TX + 4>(
        s_phi, [&](int dy, int dx) { return s_cls[dy + 3][dx + 3]; },
        [&](int dy, int dx) { return PFLBM_LD(a.wet, (y0 + dy) * pitch + wx(x0 + dx), a.plane); }, tid, TX * TY);
    __syncthreads();
}

// One tile (bx, by) of one lattice: the whole time step for its nodes.
// Called by every thread of the CTA; the shared tiles are the caller's.
// VV: 0 uniform tau_f, 1 variable viscosity, 2 decided by a.varvisc.
// WRAP: the tile or its halo of three crosses the periodic seam in x.
template <int PREC, bool COLLIDE, int VV, bool WRAP>
__device__ __forceinline__ void step_tile_w(const StepArgs<PREC>& a, int bx, int by, int ntx,
                                            uint8_t (*s_cls)[TX + 6], typename Store<PREC>::C (*s_phi)[TX + 4])
{
    using T = Store<PREC>;
    using C = typename T::C;
    const int x0 = bx * TX, y0 = by * TY;
    C g[9], f[9];
    typename T::G0T g0raw;
    const bool fluid_tile = a.tiles[by * ntx + bx] != 0;
    if (fluid_tile)
        tile_prologue_fluid<PREC, WRAP>(a, s_phi, x0, y0, g, g0raw, f);
    else
        tile_prologue<PREC, WRAP>(a, s_cls, s_phi, x0, y0, g, g0raw, f);

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int gx = x0 + tx, gy = y0 + ty;
    if (gx >= a.nx || gy >= a.ny) return;
    const uint8_t code = fluid_tile ? (uint8_t)CLS_FLUID : s_cls[ty + 3][tx + 3];
    node_step<PREC, COLLIDE, VV, TX + 4>(a, code, s_phi, ty + 2, tx + 2, gx, gy, g, g0raw, [&](C fv[9]) {
        if (PFLBM_PREFETCH_F_WALL && !fluid_tile) {
#pragma unroll
            for (int i = 0; i < 9; ++i) fv[i] = f[i];
        } else if (!fluid_tile && has_link(code))
            pull_f<PREC, true, WRAP>(fv, a.in.f, s_cls, ty + 3, tx + 3, gx, gy, a.nx, a.pitch, a.plane);
        else if (PFLBM_PREFETCH_F && fluid_tile) {
#pragma unroll
            for (int i = 0; i < 9; ++i) fv[i] = f[i];
        } else
            pull_f<PREC, false, WRAP>(fv, a.in.f, s_cls, ty + 3, tx + 3, gx, gy, a.nx, a.pitch, a.plane);
    }, [&](int k) { return (C)PFLBM_LD(a.sprev, k, a.plane); });
}

template <int PREC, bool COLLIDE, int VV>
__device__ __forceinline__ void step_tile(const StepArgs<PREC>& a, int bx, int by, int ntx,
                                          uint8_t (*s_cls)[TX + 6], typename Store<PREC>::C (*s_phi)[TX + 4])
{
    // every x the tile touches (class tile: three out) lies inside the lattice
    const int x0 = bx * TX;
    if (x0 >= 3 && x0 + TX + 3 <= a.nx)
        step_tile_w<PREC, COLLIDE, VV, false>(a, bx, by, ntx, s_cls, s_phi);
    else
        step_tile_w<PREC, COLLIDE, VV, true>(a, bx, by, ntx, s_cls, s_phi);
}

// L2 prefetch of the rows that a later tile reads: the 18 population planes
// (g_0 storage included), the u.grad(phi) history and the node bytes. The
// target is PFLBM_L2_AHEAD CTAs later in launch order, (pf_dx, pf_dy) tiles
// from this one. One row segment per thread; a segment of 32 nodes is at
// most 128 B and starts on a 128 B line (FP32 and 16-bit storage; x0 is a
// multiple of 32 and the pitch of 64). Every address lies inside the
// lattice's arrays: the tile exists and y < ny; offsets stay below
// 18 * plane < 2^31.
template <int PREC>
__device__ __forceinline__ void prefetch_tile_l2(const StepArgs<PREC>& a, int bx, int by, int ntx, int nty)
{
    static_assert(TY == 8, "one row of the tile per thread of an 8-thread group");
    if (PREC == PFLBM_FP64) return;
    int px = bx + a.pf_dx, py = by + a.pf_dy;
    if (px >= ntx) { px -= ntx; ++py; }
    const int tid = threadIdx.y * TX + threadIdx.x;
    const int q = tid >> 3, gy = py * TY + (tid & 7);
    if (py >= nty || q >= 20 || gy >= a.ny) return;
    const int row = gy * a.pitch + px * TX;
    const void* p;
    if (q < 18) {
        // FP32: g_0 is g plane 0, plane 9 of the buffer; 16-bit: its own array
        if (PREC == PFLBM_FP32 || q != 9) p = a.in.f + (q * a.plane + row);
        else p = a.in.g0 + row;
    } else if (q == 18) {
        if (a.dgdt) return;
        p = a.sprev + row;
    } else {
        if (a.tiles[py * ntx + px]) return;     // an all-fluid tile does not read its node bytes
        p = a.cls + row;
    }
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

template <int PREC, bool COLLIDE, int VV>
__global__ void __launch_bounds__(TX * TY, PREC == PFLBM_FP64 ? 1 : PFLBM_STEP_MINB) k_step(StepArgs<PREC> a)
{
    __shared__ uint8_t s_cls[TY + 6][TX + 6];
    __shared__ typename Store<PREC>::C s_phi[TY + 4][TX + 4];
    if (COLLIDE && PFLBM_L2_AHEAD > 0) prefetch_tile_l2<PREC>(a, blockIdx.x, blockIdx.y, gridDim.x, gridDim.y);
    step_tile<PREC, COLLIDE, VV>(a, blockIdx.x, blockIdx.y, gridDim.x, s_cls, s_phi);
}

// Persistent step over many lattices: work item w = (instance, first tile);
// an item covers `group` tiles of one tile column, top to bottom. CTAs take
// items w = blockIdx.x, blockIdx.x + gridDim.x, ...
template <int PREC>
__global__ void __launch_bounds__(TX * TY, PREC == PFLBM_FP64 ? 3 : PFLBM_BATCH_MINB) k_step_batch(const StepArgs<PREC>* __restrict__ args,
                                                        const int2* __restrict__ work, int n_work, int group)
{
    __shared__ uint8_t s_cls[TY + 6][TX + 6];
    __shared__ typename Store<PREC>::C s_phi[TY + 4][TX + 4];
    // the item's lattice descriptor lives in shared memory (read field by
    // field where used) rather than in registers
    __shared__ __align__(16) unsigned char s_args_raw[sizeof(StepArgs<PREC>)];
    const StepArgs<PREC>& a = *reinterpret_cast<const StepArgs<PREC>*>(s_args_raw);
    const int tid = threadIdx.y * TX + threadIdx.x;
    for (int w = blockIdx.x; w < n_work; w += gridDim.x) {
        const int2 it = work[w];
        {
            const int* src = reinterpret_cast<const int*>(args + it.x);
            int* dst = reinterpret_cast<int*>(s_args_raw);
            for (int i = tid; i < (int)(sizeof(StepArgs<PREC>) / sizeof(int)); i += TX * TY) dst[i] = src[i];
        }
        __syncthreads();
        const int ntx = tiles_x(a.nx), nty = tiles_y(a.ny);
        const int bx = it.y % ntx, by0 = it.y / ntx;
        for (int gi = 0; gi < group && by0 + gi < nty; ++gi) {
            step_tile<PREC, true, 2>(a, bx, by0 + gi, ntx, s_cls, s_phi);
            __syncthreads();   // the next tile reuses the shared tiles and descriptor
        }
    }
}

template <int PREC>
StepArgs<PREC> make_args(pflbm_t* h)
{
    using C = typename Store<PREC>::C;
    StepArgs<PREC> a{};
    const size_t plane = (size_t)h->ny * h->pitch;
    a.cls = h->cls;
    a.tiles = h->tiles;
    a.wet = (const C*)h->wet;
    a.in = Planes<PREC>::make(h->pop[h->cur], plane);
    a.out = Planes<PREC>::make(h->pop[h->cur ^ 1], plane);
    a.sprev = (C*)h->sprev;
    a.nx = h->nx;
    a.ny = h->ny;
    a.pitch = h->pitch;
    a.plane = (int)plane;
    const Params& q = h->prm;
    a.beta4 = (C)(4.0 * q.beta);
    a.kappa = (C)q.kappa;
    a.rho_g = (C)q.rho_g;
    a.drho = (C)(q.rho_l - q.rho_g);
    a.omega_f = (C)(1.0 / q.tau_f);
    a.omega_g = (C)(1.0 / q.tau_g);
    a.force_pre = (C)(1.0 - 1.0 / (2.0 * q.tau_f));
    a.alpha = (C)q.alpha;
    a.varvisc = (q.nu_l > 0 && q.nu_g > 0) ? 1 : 0;
    a.pf_dx = PFLBM_L2_AHEAD % tiles_x(h->nx);
    a.pf_dy = PFLBM_L2_AHEAD / tiles_x(h->nx);
    a.dgdt = q.dgdt_mode;
    a.tau_g3h = (C)(3.0 * q.nu_g + 0.5);
    a.dtau3 = (C)(3.0 * (q.nu_l - q.nu_g));
    a.gx = (C)q.gx;
    a.gy = (C)q.gy;
    a.status = h->dstatus;
    a.tma = h->tma;
    a.in_copy = h->cur;
    a.sflags[0] = h->sflags;
    a.sflags[1] = h->sflags ? h->sflags + (size_t)((h->nx + 31) / 32) * ((h->ny + 7) / 8) : nullptr;
    a.nword = h->nword;
    a.tiles2 = h->tiles2;
    return a;
}

// ---------------------------------------------------------------------------
// Initial state (FP64 arithmetic for every storage precision)
// ---------------------------------------------------------------------------
// Eq. initialphi over the box x in [xlo, xlo + xw) (x periodic), y in
// [ylo, yhi), combined with the field by maximum (a replacing call cleared it).
// F32: the profile in FP32 (solves whose arithmetic is FP32 or 16-bit storage;
// the FP64 tanh is slow on this part), else in FP64.
template <bool F32>
__global__ void k_init_droplet(const uint8_t* __restrict__ cls, double* __restrict__ phi, int nx, int ny,
                               int pitch, int xlo, int xw, int ylo, int yhi, double x0, double y0, double R,
                               double W)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int y = ylo + blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= xw || y >= yhi) return;
    int x = (xlo + i) % nx;
    if (x < 0) x += nx;
    size_t k = (size_t)y * pitch + x;
    if (!zeta_of(cls[k])) return;
    double dx = fabs((double)x - x0);
    if (dx >= nx) dx = fmod(dx, (double)nx);   // exact; only for a period or more
    if (dx > 0.5 * nx) dx = nx - dx;           // x-periodic distance
    const double dy = (double)y - y0, r2 = dx * dx + dy * dy;
    // beyond |R| + 10 W the profile is 0 in FP64 (tanh(-20) rounds to -1):
    // the bounding box's corners are skipped like the nodes outside it
    const double reach = fabs(R) + 10.0 * W;
    if (r2 > reach * reach) return;
    const double v = F32 ? (double)(0.5f + 0.5f * tanhf(2.0f * ((float)R - sqrtf((float)r2)) / (float)W))
                         : 0.5 + 0.5 * tanh(2.0 * (R - sqrt(r2)) / W);
    if (v > phi[k]) phi[k] = v;
}

template <typename C>
__global__ void k_ghost_fill(const uint8_t* __restrict__ cls, const C* __restrict__ wet, double* __restrict__ phi,
                             int nx, int ny, int pitch)
{
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= nx || y >= ny) return;
    size_t k = (size_t)y * pitch + x;
    const uint8_t code = cls[k];
    uint8_t c = code & CLS_MASK;
    if (c == CLS_INTERIOR) { phi[k] = 0.0; return; }
    if (c != CLS_GHOST) return;
    if (code & (F_GHOST_UP | F_GHOST_DOWN)) {
        // the mirror node is zeta = 1, never a ghost: no ordering hazard
        phi[k] = robin_ghost<double>(phi[(code & F_GHOST_UP) ? k + pitch : k - pitch], (double)wet[k]);
        return;
    }
    double num = 0.0, den = 0.0;
    for (int j = 1; j < 9; ++j) {
        int yy = y + cy(j);
        if (yy < 0 || yy >= ny) continue;
        size_t m = (size_t)yy * pitch + wrap1(x + cx(j), nx);
        if (zeta_of(cls[m])) { num += phi[m]; den += 1.0; }
    }
    phi[k] = num / den;
}

template <typename C>
__global__ void k_init_mu(const uint8_t* __restrict__ cls, const C* __restrict__ wet, const double* __restrict__ phi,
                          double* __restrict__ mu, C* __restrict__ sprev, int nx, int ny, int pitch, Params q)
{
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= nx || y >= ny) return;
    size_t k = (size_t)y * pitch + x;
    uint8_t code = cls[k];
    if (!zeta_of(code)) { mu[k] = 0.0; sprev[k] = (C)0; return; }
    // in the precision of the step's arithmetic (C): FP64 for FP64 solves,
    // FP32 otherwise (FP64 arithmetic is slow on this part, and a 32-bit
    // state stores mu only through g_i^eq = w_i alpha mu, rounded to 32 or
    // 16 bits; phi = sum g_i stays exact through g_0)
    auto at = [&](int dx, int dy) { return (C)phi[(size_t)(y + dy) * pitch + wrap1(x + dx, nx)]; };
    const C c = (C)phi[k];
    const C E = at(1, 0), Wv = at(-1, 0), N = at(0, 1), S = at(0, -1);
    const C NE = at(1, 1), NW = at(-1, 1), SW = at(-1, -1), SE = at(1, -1);
    // multiplications by rounded reciprocals: division is slow
    const C gpx = (E - Wv) * (C(1) / C(3)) + ((NE + SE) - (NW + SW)) * (C(1) / C(12));
    const C gpy = (N - S) * (C(1) / C(3)) + ((NE + NW) - (SE + SW)) * (C(1) / C(12));
    const C lap = ((E + Wv) + (N + S)) * (C(2) / C(3)) + ((NE + NW) + (SE + SW)) * (C(1) / C(6)) - c * (C(10) / C(3));
    const C wv = (code & F_WET) ? wet[k] : C(0);
    const C m = C(4) * (C)q.beta * c * (c - C(1)) * (c - C(0.5)) - (C)q.kappa * lap - wv * (c - c * c);
    mu[k] = (double)m;
    // u at t = 0 from f = 0: u = F / (2 rho), F = mu grad(phi) + rho g; the
    // history of the first step is u.grad(phi)
    const C rho = (C)q.rho_g + (C)(q.rho_l - q.rho_g) * c;
    const C half_inv_rho = C(0.5) / rho;
    const C ux = (m * gpx + rho * (C)q.gx) * half_inv_rho, uy = (m * gpy + rho * (C)q.gy) * half_inv_rho;
    sprev[k] = ux * gpx + uy * gpy;
}

// g_J^eq (J != 0) in storage form; returns the rounding residual.
template <int PREC, int J>
__device__ __forceinline__ double init_g_dir(const uint8_t* cls, const double* mu, const Planes<PREC>& P, int x,
                                             int y, int nx, int pitch, size_t k, size_t plane, double alpha)
{
    using T = Store<PREC>;
    // the pull at x + c_j reads this value as its g_j when x + c_j is a
    // zeta = 1 node; when it is not, only the doubly-unknown rule of this
    // node reads it, as the node's own value
    size_t m = (size_t)(y + cy(J)) * pitch + wrap1(x + cx(J), nx);
    if (!zeta_of(cls[m])) m = k;
    const double w = J <= 4 ? 1.0 / 9.0 : 1.0 / 36.0;
    const double v = w * alpha * mu[m];
    const typename T::S s = T::template st<J>((typename T::C)v);
    P.g[J * plane + k] = s;
    return v - (double)T::template ld<J>(s);
}

// Post-collision arrays that the first pull turns into f = 0, g = g^eq(phi0, mu0).
template <int PREC>
__global__ void k_init_pop(const uint8_t* __restrict__ cls, const double* __restrict__ phi,
                           const double* __restrict__ mu, Planes<PREC> P, int nx, int ny, int pitch, size_t plane,
                           double alpha)
{
    using T = Store<PREC>;
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= nx || y >= ny) return;
    size_t k = (size_t)y * pitch + x;
    const typename T::S zero = T::template st<0>((typename T::C)0);
    for (int i = 0; i < 9; ++i) {
        P.f[i * plane + k] = zero;
        P.g[i * plane + k] = zero;
    }
    P.g0[k] = T::g0_from_double(0.0);
    if (!zeta_of(cls[k])) return;
    double r = 0.0;
    r += init_g_dir<PREC, 1>(cls, mu, P, x, y, nx, pitch, k, plane, alpha);
    r += init_g_dir<PREC, 2>(cls, mu, P, x, y, nx, pitch, k, plane, alpha);
    r += init_g_dir<PREC, 3>(cls, mu, P, x, y, nx, pitch, k, plane, alpha);
    r += init_g_dir<PREC, 4>(cls, mu, P, x, y, nx, pitch, k, plane, alpha);
    r += init_g_dir<PREC, 5>(cls, mu, P, x, y, nx, pitch, k, plane, alpha);
    r += init_g_dir<PREC, 6>(cls, mu, P, x, y, nx, pitch, k, plane, alpha);
    r += init_g_dir<PREC, 7>(cls, mu, P, x, y, nx, pitch, k, plane, alpha);
    r += init_g_dir<PREC, 8>(cls, mu, P, x, y, nx, pitch, k, plane, alpha);
    // g_0^eq (Eq. H_i); with 16-bit g_i it also holds their rounding residual
    double g0 = phi[k] - (5.0 / 9.0) * alpha * mu[k];
    if (T::kAbsorb) g0 += r;
    P.g0[k] = T::g0_from_double(g0);
}

dim3 grid2d(int nx, int ny, dim3 b) { return dim3((nx + b.x - 1) / b.x, (ny + b.y - 1) / b.y); }

template <int PREC, bool COLLIDE>
cudaError_t run_step_kernel(pflbm_t* h, double* o_phi, double* o_u, double* o_p, float* f_phi = nullptr,
                            float* f_u = nullptr, float* f_p = nullptr)
{
    StepArgs<PREC> a = make_args<PREC>(h);
    a.o_phi = o_phi;
    a.o_u = o_u;
    a.o_p = o_p;
    a.f_phi = f_phi;
    a.f_u = f_u;
    a.f_p = f_p;
    dim3 b(TX, TY), g(tiles_x(h->nx), tiles_y(h->ny));
    if (a.varvisc)
        k_step<PREC, COLLIDE, 1><<<g, b, 0, h->stream>>>(a);
    else
        k_step<PREC, COLLIDE, 0><<<g, b, 0, h->stream>>>(a);
    return cudaGetLastError();
}

template <int PREC>
cudaError_t init_pop_prec(pflbm_t* h)
{
    using C = typename Store<PREC>::C;
    dim3 b(32, 8), g = grid2d(h->nx, h->ny, b);
    size_t plane = (size_t)h->ny * h->pitch;
    k_init_mu<C><<<g, b, 0, h->stream>>>(h->cls, (const C*)h->wet, h->phi0, h->mu0, (C*)h->sprev, h->nx, h->ny,
                                         h->pitch, h->prm);
    k_init_pop<PREC><<<g, b, 0, h->stream>>>(h->cls, h->phi0, h->mu0, Planes<PREC>::make(h->pop[h->cur], plane),
                                             h->nx, h->ny, h->pitch, plane, h->prm.alpha);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_init_phi_droplet(pflbm_t* h, double x0, double y0, double R, int replace)
{
    // Outside r = R + 10 W the profile is exactly 0 in FP64 (tanh(-20) rounds
    // to -1), so only the droplet's bounding box is evaluated; a replacing
    // call clears the field first.
    if (replace) {
        cudaError_t e = cudaMemsetAsync(h->phi0, 0, (size_t)h->ny * h->pitch * sizeof(double), h->stream);
        if (e != cudaSuccess) return e;
    }
    double reach = fabs(R) + 10.0 * h->prm.W;
    int ylo = (int)fmax(0.0, floor(y0 - reach)), yhi = (int)fmin((double)h->ny - 1, ceil(y0 + reach));
    if (ylo > yhi) return cudaSuccess;
    int xlo = 0, xw = h->nx;
    if (2.0 * reach + 2.0 < h->nx) {
        xlo = (int)floor(x0 - reach);
        xw = (int)(ceil(x0 + reach) - floor(x0 - reach)) + 1;
    }
    dim3 b(32, 8), g = grid2d(xw, yhi - ylo + 1, b);
    if (h->precision == PFLBM_FP64)
        k_init_droplet<false><<<g, b, 0, h->stream>>>(h->cls, h->phi0, h->nx, h->ny, h->pitch, xlo, xw, ylo, yhi + 1,
                                                      x0, y0, R, h->prm.W);
    else
        k_init_droplet<true><<<g, b, 0, h->stream>>>(h->cls, h->phi0, h->nx, h->ny, h->pitch, xlo, xw, ylo, yhi + 1,
                                                     x0, y0, R, h->prm.W);
    return cudaGetLastError();
}

cudaError_t launch_init_populations(pflbm_t* h)
{
    dim3 b(32, 8), g = grid2d(h->nx, h->ny, b);
    if (h->precision == PFLBM_FP64)
        k_ghost_fill<double><<<g, b, 0, h->stream>>>(h->cls, (const double*)h->wet, h->phi0, h->nx, h->ny, h->pitch);
    else
        k_ghost_fill<float><<<g, b, 0, h->stream>>>(h->cls, (const float*)h->wet, h->phi0, h->nx, h->ny, h->pitch);
    switch (h->precision) {
        case PFLBM_FP64: return init_pop_prec<PFLBM_FP64>(h);
        case PFLBM_FP32: return init_pop_prec<PFLBM_FP32>(h);
        case PFLBM_BF16: return init_pop_prec<PFLBM_BF16>(h);
        default: return init_pop_prec<PFLBM_FP16>(h);
    }
}

cudaError_t launch_step(pflbm_t* h)
{
    cudaError_t e;
    if (h->tma && h->step_shape >= 0 && h->precision != PFLBM_FP64) {
        e = launch_step_staged(h, h->step_shape, h->step_chunk, 0);
        if (e == cudaSuccess) h->cur ^= 1;
        return e;
    }
    if (h->step_shape == -2 && h->precision != PFLBM_FP64) {
        e = launch_step2(h);
        if (e == cudaSuccess) h->cur ^= 1;
        return e;
    }
    switch (h->precision) {
        case PFLBM_FP64: e = run_step_kernel<PFLBM_FP64, true>(h, nullptr, nullptr, nullptr); break;
        case PFLBM_FP32: e = run_step_kernel<PFLBM_FP32, true>(h, nullptr, nullptr, nullptr); break;
        case PFLBM_BF16: e = run_step_kernel<PFLBM_BF16, true>(h, nullptr, nullptr, nullptr); break;
        default: e = run_step_kernel<PFLBM_FP16, true>(h, nullptr, nullptr, nullptr); break;
    }
    if (e == cudaSuccess) h->cur ^= 1;
    return e;
}

size_t step_args_bytes(int precision)
{
    switch (precision) {
        case PFLBM_FP64: return sizeof(StepArgs<PFLBM_FP64>);
        case PFLBM_FP32: return sizeof(StepArgs<PFLBM_FP32>);
        case PFLBM_BF16: return sizeof(StepArgs<PFLBM_BF16>);
        default: return sizeof(StepArgs<PFLBM_FP16>);
    }
}

namespace {
template <int PREC>
void write_args_prec(pflbm_t* h, int flip, void* dst)
{
    StepArgs<PREC> a = make_args<PREC>(h);
    if (flip) {
        Planes<PREC> t = a.in;
        a.in = a.out;
        a.out = t;
        a.in_copy ^= 1;
    }
    *(StepArgs<PREC>*)dst = a;
}
}  // namespace

void write_step_args(pflbm_t* h, int flip, void* dst)
{
    switch (h->precision) {
        case PFLBM_FP64: write_args_prec<PFLBM_FP64>(h, flip, dst); break;
        case PFLBM_FP32: write_args_prec<PFLBM_FP32>(h, flip, dst); break;
        case PFLBM_BF16: write_args_prec<PFLBM_BF16>(h, flip, dst); break;
        default: write_args_prec<PFLBM_FP16>(h, flip, dst); break;
    }
}

cudaError_t launch_step_batch(int precision, const void* d_args, const int2* d_work, int n_work, int group,
                              int grid, cudaStream_t stream)
{
    dim3 b(TX, TY);
    switch (precision) {
        case PFLBM_FP64:
            k_step_batch<PFLBM_FP64><<<grid, b, 0, stream>>>((const StepArgs<PFLBM_FP64>*)d_args, d_work, n_work, group);
            break;
        case PFLBM_FP32:
            k_step_batch<PFLBM_FP32><<<grid, b, 0, stream>>>((const StepArgs<PFLBM_FP32>*)d_args, d_work, n_work, group);
            break;
        case PFLBM_BF16:
            k_step_batch<PFLBM_BF16><<<grid, b, 0, stream>>>((const StepArgs<PFLBM_BF16>*)d_args, d_work, n_work, group);
            break;
        default:
            k_step_batch<PFLBM_FP16><<<grid, b, 0, stream>>>((const StepArgs<PFLBM_FP16>*)d_args, d_work, n_work, group);
            break;
    }
    return cudaGetLastError();
}

int batch_max_ctas_per_sm(int precision)
{
    int n = 0;
    cudaError_t e;
    switch (precision) {
        case PFLBM_FP64: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_batch<PFLBM_FP64>, TX * TY, 0); break;
        case PFLBM_FP32: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_batch<PFLBM_FP32>, TX * TY, 0); break;
        case PFLBM_BF16: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_batch<PFLBM_BF16>, TX * TY, 0); break;
        default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_batch<PFLBM_FP16>, TX * TY, 0); break;
    }
    return e == cudaSuccess ? n : 1;
}

cudaError_t launch_macro(pflbm_t* h, double* phi, double* u, double* p)
{
    switch (h->precision) {
        case PFLBM_FP64: return run_step_kernel<PFLBM_FP64, false>(h, phi, u, p);
        case PFLBM_FP32: return run_step_kernel<PFLBM_FP32, false>(h, phi, u, p);
        case PFLBM_BF16: return run_step_kernel<PFLBM_BF16, false>(h, phi, u, p);
        default: return run_step_kernel<PFLBM_FP16, false>(h, phi, u, p);
    }
}

cudaError_t launch_macro_f32(pflbm_t* h, float* phi, float* u, float* p)
{
    switch (h->precision) {
        case PFLBM_FP64: return run_step_kernel<PFLBM_FP64, false>(h, nullptr, nullptr, nullptr, phi, u, p);
        case PFLBM_FP32: return run_step_kernel<PFLBM_FP32, false>(h, nullptr, nullptr, nullptr, phi, u, p);
        case PFLBM_BF16: return run_step_kernel<PFLBM_BF16, false>(h, nullptr, nullptr, nullptr, phi, u, p);
        default: return run_step_kernel<PFLBM_FP16, false>(h, nullptr, nullptr, nullptr, phi, u, p);
    }
}

#ifdef PFLBM_BOUNDS
unsigned bounds_violations_step()
{
    unsigned v = 0;
    cudaMemcpyFromSymbol(&v, g_bounds_viol, sizeof(v));
    return v;
}
#else
unsigned bounds_violations_step() { return 0; }
#endif

}  // namespace pfk
