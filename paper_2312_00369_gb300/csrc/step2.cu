// step2.cu -- the time step with two x-adjacent nodes per thread, in packed
// FP32x2 arithmetic (FP32 and 16-bit storage).
//
// A CTA of 32 x 8 threads takes a 64 x 8 tile: thread (tx, ty) owns the
// nodes x0 + 2 tx and x0 + 2 tx + 1 of row y0 + ty. The prologue is that of
// the one-node kernel on a wider tile (phi tile with a ring of one, or two
// next to ghosts; ghost values; bounce-back pulls decided per warp), and the
// per-node arithmetic is node_core (step_core.cuh) on F2 lanes: every
// operation of the two nodes is one packed instruction (add/sub/mul/fma.rn
// on .f32x2), each lane rounding exactly as the scalar code, so
// the results equal the one-node kernel's bit for bit. The two nodes' values
// leave as one 32-bit (16-bit storage) or 64-bit (FP32) store per plane, and
// on tiles away from the periodic seam the pulls of the directions without
// an x component are one aligned load for both nodes.
#include "step_core.cuh"

#include <type_traits>

namespace pfk {
namespace {

constexpr int QX = 64, QY = 8;        // tile (nodes)
constexpr int QTX = QX / 2;           // threads in x
constexpr int QCW = QX + 6;           // class tile row (halo 3)
constexpr int QPW = QX + 4;           // phi tile row (halo 2)

// L2 prefetch distance in CTAs of launch order (0: off): a quarter of the
// 3 x 152 resident CTAs, the same node distance as the one-node kernel's
// single-lattice kernel, fluid tiles: pull f with g, before the phi-tile
// barrier (twice the loads in flight per thread, for 9 more registers;
// measured faster there, slower in the batched kernel, which spills)
#ifndef PFLBM_PAIR_EARLY_F
#define PFLBM_PAIR_EARLY_F 1
#endif

// resident 256-thread CTAs per SM asked of k_step2: 4 with 16-bit storage
// (64 registers, the pulled populations held as raw pairs), 3 with FP32
#ifndef PFLBM_STEP2_MINB
#define PFLBM_STEP2_MINB 4
#endif
#ifndef PFLBM_STEP2_MINB32
#define PFLBM_STEP2_MINB32 3
#endif
#ifndef PFLBM_L2_AHEAD2
#define PFLBM_L2_AHEAD2 114
#endif

// Pull of direction I for the two nodes (gx, gy), (gx + 1, gy), gx even,
// from neighbours that are all zeta = 1 (no bounce-back).
template <int I, int PREC, bool WRAP>
__device__ __forceinline__ F2 pull2(const typename Store<PREC>::S* __restrict__ base, int gx, int gy, int nx,
                                    int pitch, int plane)
{
    using T = Store<PREC>;
    constexpr int X = cx(I), Y = cy(I);
    if constexpr (!WRAP) {
        const int idx = gy * pitch + gx + (I * plane - Y * pitch - X);
        if constexpr (X == 0) {
            // aligned pair: gx is even and every plane and row starts on an
            // even element
            if constexpr (PREC == PFLBM_FP32) {
                const float2 v = PFLBM_LD(reinterpret_cast<const float2*>(base), idx / 2, 9LL * plane / 2);
                return F2(v.x, v.y);
            } else {
                const uint32_t u = PFLBM_LD(reinterpret_cast<const uint32_t*>(base), idx / 2, 9LL * plane / 2);
                typename T::S lo, hi;
                const uint16_t l16 = (uint16_t)(u & 0xffffu), h16 = (uint16_t)(u >> 16);
                memcpy(&lo, &l16, 2);
                memcpy(&hi, &h16, 2);
                return F2(T::template ldp<I>(lo), T::template ldp<I>(hi));
            }
        } else {
            return F2(T::template ldp<I>(PFLBM_LD(base, idx, 9LL * plane)),
                      T::template ldp<I>(PFLBM_LD(base, idx + 1, 9LL * plane)));
        }
    } else {
        const int r = (gy - Y) * pitch + I * plane;
        return F2(T::template ldp<I>(PFLBM_LD(base, r + wrap1(gx - X, nx), 9LL * plane)),
                  T::template ldp<I>(PFLBM_LD(base, r + wrap1(gx + 1 - X, nx), 9LL * plane)));
    }
}

// The same for 16-bit storage, as the raw pair (lane x in the low half):
// the aligned word itself for directions without an x component away from
// the seam, else two 16-bit loads joined.
template <int I, int PREC, bool WRAP>
__device__ __forceinline__ uint32_t pull2_raw(const typename Store<PREC>::S* __restrict__ base, int gx, int gy, int nx,
                                              int pitch, int plane)
{
    static_assert(PREC != PFLBM_FP32, "16-bit storage");
    constexpr int X = cx(I), Y = cy(I);
    const uint16_t* b = reinterpret_cast<const uint16_t*>(base);
    if constexpr (!WRAP) {
        const int idx = gy * pitch + gx + (I * plane - Y * pitch - X);
        if constexpr (X == 0)
            return PFLBM_LD(reinterpret_cast<const uint32_t*>(base), idx / 2, 9LL * plane / 2);
        else
            return (uint32_t)PFLBM_LD(b, idx, 9LL * plane) | ((uint32_t)PFLBM_LD(b, idx + 1, 9LL * plane) << 16);
    } else {
        const int r = (gy - Y) * pitch + I * plane;
        return (uint32_t)PFLBM_LD(b, r + wrap1(gx - X, nx), 9LL * plane) |
               ((uint32_t)PFLBM_LD(b, r + wrap1(gx + 1 - X, nx), 9LL * plane) << 16);
    }
}


template <int I, int PREC, bool WRAP>
__device__ __forceinline__ typename Hold2<PREC>::W pull2_w(const typename Store<PREC>::S* __restrict__ base, int gx,
                                                        int gy, int nx, int pitch, int plane)
{
    if constexpr (Hold2<PREC>::kRaw) return pull2_raw<I, PREC, WRAP>(base, gx, gy, nx, pitch, plane);
    else return pull2<I, PREC, WRAP>(base, gx, gy, nx, pitch, plane);
}

template <int PREC, bool WRAP>
__device__ __forceinline__ void pull2_f(Hold2<PREC>& v, const typename Store<PREC>::S* __restrict__ f, int gx, int gy,
                                        int nx, int pitch, int plane)
{
    v.w[0] = pull2_w<0, PREC, WRAP>(f, gx, gy, nx, pitch, plane);
    v.w[1] = pull2_w<1, PREC, WRAP>(f, gx, gy, nx, pitch, plane);
    v.w[2] = pull2_w<2, PREC, WRAP>(f, gx, gy, nx, pitch, plane);
    v.w[3] = pull2_w<3, PREC, WRAP>(f, gx, gy, nx, pitch, plane);
    v.w[4] = pull2_w<4, PREC, WRAP>(f, gx, gy, nx, pitch, plane);
    v.w[5] = pull2_w<5, PREC, WRAP>(f, gx, gy, nx, pitch, plane);
    v.w[6] = pull2_w<6, PREC, WRAP>(f, gx, gy, nx, pitch, plane);
    v.w[7] = pull2_w<7, PREC, WRAP>(f, gx, gy, nx, pitch, plane);
    v.w[8] = pull2_w<8, PREC, WRAP>(f, gx, gy, nx, pitch, plane);
}

// g of the two nodes (no bounce-back) and their raw g_0 (an aligned pair).
template <int PREC, bool WRAP>
__device__ __forceinline__ void pull2_g(Hold2<PREC>& v, int32_t raw[2], const Planes<PREC>& P, int gx, int gy, int nx,
                                        int pitch, int plane)
{
    if constexpr (!WRAP) {
        const int2 r = PFLBM_LD(reinterpret_cast<const int2*>(P.g0), (gy * pitch + gx) / 2, plane / 2);
        raw[0] = r.x;
        raw[1] = r.y;
    } else {
        raw[0] = PFLBM_LD(P.g0, gy * pitch + wrap1(gx, nx), plane);
        raw[1] = PFLBM_LD(P.g0, gy * pitch + wrap1(gx + 1, nx), plane);
    }
    v.w[1] = pull2_w<1, PREC, WRAP>(P.g, gx, gy, nx, pitch, plane);
    v.w[2] = pull2_w<2, PREC, WRAP>(P.g, gx, gy, nx, pitch, plane);
    v.w[3] = pull2_w<3, PREC, WRAP>(P.g, gx, gy, nx, pitch, plane);
    v.w[4] = pull2_w<4, PREC, WRAP>(P.g, gx, gy, nx, pitch, plane);
    v.w[5] = pull2_w<5, PREC, WRAP>(P.g, gx, gy, nx, pitch, plane);
    v.w[6] = pull2_w<6, PREC, WRAP>(P.g, gx, gy, nx, pitch, plane);
    v.w[7] = pull2_w<7, PREC, WRAP>(P.g, gx, gy, nx, pitch, plane);
    v.w[8] = pull2_w<8, PREC, WRAP>(P.g, gx, gy, nx, pitch, plane);
}

// phi = sum_i g_i (Eq. order-parameter) of both lanes, in the scalar order.
template <int PREC>
__device__ __forceinline__ F2 phi2(const Hold2<PREC>& v, const int32_t raw[2])
{
    using T = Store<PREC>;
    F2 s;
    if constexpr (T::kNorm)
        s = fmadd(F2(T::template unit<1>()), (v[1] + v[2]) + (v[3] + v[4]),
                  F2(T::template unit<5>()) * ((v[5] + v[6]) + (v[7] + v[8])));
    else
        s = ((v[1] + v[2]) + (v[3] + v[4])) + ((v[5] + v[6]) + (v[7] + v[8]));
    return F2(T::g0(raw[0]), T::g0(raw[1])) + s;
}

// Ring positions (width H) around the 64 x 8 tile: phi of one node each.
template <int PREC, int H, bool WRAP, bool FLUID>
__device__ __forceinline__ void ring2(const StepArgs<PREC>& a, const uint8_t (*s_cls)[QCW], float (*s_phi)[QPW], int x0,
                                      int y0, int tid, bool tiny)
{
    constexpr int RW = QX + 2 * H, NTOP = H * RW, NSIDE = H * QY, NR = 2 * NTOP + 2 * NSIDE;
    for (int t = tid; t < NR; t += QTX * QY) {
        int py, px;
        if (t < NTOP) { py = 2 - H + t / RW; px = 2 - H + t % RW; }
        else if (t < 2 * NTOP) { const int u = t - NTOP; py = QY + 2 + u / RW; px = 2 - H + u % RW; }
        else if (t < 2 * NTOP + NSIDE) { const int u = t - 2 * NTOP; py = 2 + u / H; px = 2 - H + u % H; }
        else { const int u = t - 2 * NTOP - NSIDE; py = 2 + u / H; px = QX + 2 + u % H; }
        const int gy = y0 - 2 + py, xr = x0 - 2 + px;
        const int gx = !WRAP ? xr : (tiny ? wrapn(xr, a.nx) : wrap1(xr, a.nx));
        float ph = 0.0f;
        if (FLUID) {
            ph = pulled_phi<PREC, false, WRAP, QCW>(a.in, nullptr, 0, 0, gx, gy, a.nx, a.pitch, a.plane);
        } else {
            const int sy = py + 1, sx = px + 1;
            const uint8_t c = s_cls[sy][sx];
            if (zeta_of(c)) {
                if (has_link(c))
                    ph = pulled_phi<PREC, true, WRAP, QCW>(a.in, s_cls, sy, sx, gx, gy, a.nx, a.pitch, a.plane);
                else
                    ph = pulled_phi<PREC, false, WRAP, QCW>(a.in, s_cls, sy, sx, gx, gy, a.nx, a.pitch, a.plane);
            }
        }
        s_phi[py][px] = ph;
    }
}

// One scalar node's g (with bounce-back when it has an unknown link).
template <int PREC, bool WRAP>
__device__ __forceinline__ float own_g(float v[9], int32_t& raw, const StepArgs<PREC>& a, const uint8_t (*s_cls)[QCW],
                                       int sy, int sx, int gx, int gy, uint8_t code)
{
    if (has_link(code))
        pull_g<PREC, true, WRAP, QCW>(v, raw, a.in, s_cls, sy, sx, gx, gy, a.nx, a.pitch, a.plane);
    else
        pull_g<PREC, false, WRAP, QCW>(v, raw, a.in, s_cls, sy, sx, gx, gy, a.nx, a.pitch, a.plane);
    return phi_of<PREC>(v);
}

template <int PREC, int VV, bool WRAP, bool EARLY_F>
__device__ __forceinline__ void tile2(const StepArgs<PREC>& a, int bx, int by, uint8_t (*s_cls)[QCW],
                                      float (*s_phi)[QPW])
{
    using T = Store<PREC>;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * QTX + tx;
    const int x0 = bx * QX, y0 = by * QY;
    const int nx = a.nx, ny = a.ny, pitch = a.pitch;
    const int ntx = tiles_x(nx);
    // the two 32 x 8 tiles of this one: fluid when both are (or the right
    // one lies beyond the lattice)
    const bool fluid = a.tiles[by * ntx + 2 * bx] != 0 && (2 * bx + 1 >= ntx || a.tiles[by * ntx + 2 * bx + 1] != 0);
    const bool tiny = nx < QX + 8;
    const int gxa = x0 + 2 * tx, gy = y0 + ty;
    Hold2<PREC> g;
    int32_t raw[2] = {0, 0};
    uint8_t code[2] = {CLS_FLUID, CLS_FLUID};

    Hold2<PREC> fearly;
    if (fluid) {
        // ---- prologue of an all-fluid tile: no class tile, no checks ----
        pull2_g<PREC, WRAP>(g, raw, a.in, gxa, gy, nx, pitch, a.plane);
        if (EARLY_F) pull2_f<PREC, WRAP>(fearly, a.in.f, gxa, gy, nx, pitch, a.plane);
        const F2 ph = phi2<PREC>(g, raw);
        s_phi[ty + 2][2 * tx + 2] = ph.x;
        s_phi[ty + 2][2 * tx + 3] = ph.y;
        ring2<PREC, 1, WRAP, true>(a, s_cls, s_phi, x0, y0, tid, tiny);
        __syncthreads();
    } else {
        // ---- general prologue: class tile (halo 3), phi tile, ghosts ----
        auto wx = [&](int x) { return !WRAP ? x : (tiny ? wrapn(x, nx) : wrap1(x, nx)); };
        for (int p = tid; p < (QY + 6) * QCW; p += QTX * QY) {
            const int py = p / QCW, px = p - py * QCW;
            const int yy = y0 - 3 + py, xx = wx(x0 - 3 + px);
            s_cls[py][px] = (yy < 0 || yy >= ny) ? (uint8_t)CLS_OUT : PFLBM_LD(a.cls, yy * pitch + xx, a.plane);
        }
        __syncthreads();
        code[0] = s_cls[ty + 3][2 * tx + 3];
        code[1] = s_cls[ty + 3][2 * tx + 4];
        bool near_ghost = false;
        for (int j = 0; j < 2; ++j) {
            const uint8_t c = code[j];
            near_ghost |= (gy < ny) && c != CLS_OUT &&
                          ((zeta_of(c) && (c & F_NEARGHOST)) || (c & CLS_MASK) == CLS_GHOST);
        }
        const int halo = __syncthreads_or(near_ghost) ? 2 : 1;
        float ga[9], gb[9];
        float pha = 0.0f, phb = 0.0f;
#pragma unroll
        for (int i = 0; i < 9; ++i) ga[i] = gb[i] = 0.0f;
        if (gy < ny && zeta_of(code[0]))
            pha = own_g<PREC, WRAP>(ga, raw[0], a, s_cls, ty + 3, 2 * tx + 3, wx(gxa), gy, code[0]);
        if (gy < ny && zeta_of(code[1]))
            phb = own_g<PREC, WRAP>(gb, raw[1], a, s_cls, ty + 3, 2 * tx + 4, wx(gxa + 1), gy, code[1]);
#pragma unroll
        for (int i = 1; i < 9; ++i) g.set(i, F2(ga[i], gb[i]));
        s_phi[ty + 2][2 * tx + 2] = pha;
        s_phi[ty + 2][2 * tx + 3] = phb;
        if (halo == 1) ring2<PREC, 1, WRAP, false>(a, s_cls, s_phi, x0, y0, tid, tiny);
        else ring2<PREC, 2, WRAP, false>(a, s_cls, s_phi, x0, y0, tid, tiny);
        __syncthreads();
        if (halo == 2) {
            fill_ghosts<float, QX, QY, QPW>(
                s_phi, [&](int dy, int dx) { return s_cls[dy + 3][dx + 3]; },
                [&](int dy, int dx) { return PFLBM_LD(a.wet, (y0 + dy) * pitch + wx(x0 + dx), a.plane); }, tid,
                QTX * QY);
            __syncthreads();
        }
    }

    // ---- the two nodes ----
    if (gy >= ny) return;
    Lane2<PREC> lane;
    lane.code[0] = code[0];
    lane.code[1] = code[1];
    lane.valid[0] = gxa < nx && zeta_of(code[0]);
    lane.valid[1] = gxa + 1 < nx && zeta_of(code[1]);
    if (!lane.valid[0] && !lane.valid[1]) return;
    lane.k = gy * pitch + gxa;
    lane.g0raw[0] = raw[0];
    lane.g0raw[1] = raw[1];
    // the 4 x 3 phi values around the pair, as three aligned float2 per row
    // (64-bit shared loads: no bank conflicts): W = (l.y, m.x), C = m, E = (m.y, r.x)
    const int py = ty + 2, px = 2 * tx + 2;
    F2 Wr[3], Cr[3], Er[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const float2* row = reinterpret_cast<const float2*>(&s_phi[py - 1 + r][0]);
        const float2 l = row[px / 2 - 1], m = row[px / 2], rr = row[px / 2 + 1];
        Wr[r] = F2(l.y, m.x);
        Cr[r] = F2(m.x, m.y);
        Er[r] = F2(m.y, rr.x);
    }
    F2 gpx, gpy, lap;
    stencil9<F2>(Cr[1], Er[1], Wr[1], Cr[2], Cr[0], Er[2], Wr[2], Wr[0], Er[0], gpx, gpy, lap);
    node_core<PREC, true, VV>(
        a, lane, Cr[1], gpx, gpy, lap, g,
        [&](Hold2<PREC>& fv) {
            if (fluid) {
                if (EARLY_F) fv = fearly;
                else pull2_f<PREC, WRAP>(fv, a.in.f, gxa, gy, nx, pitch, a.plane);
                return;
            }
            float fa[9], fb[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) fa[i] = fb[i] = 0.0f;
            auto one = [&](float v[9], int j, int gxj) {
                if (!lane.valid[j]) return;
                if (has_link(code[j]))
                    pull_f<PREC, true, WRAP, QCW>(v, a.in.f, s_cls, ty + 3, 2 * tx + 3 + j, gxj, gy, nx, pitch, a.plane);
                else
                    pull_f<PREC, false, WRAP, QCW>(v, a.in.f, s_cls, ty + 3, 2 * tx + 3 + j, gxj, gy, nx, pitch,
                                                   a.plane);
            };
            one(fa, 0, gxa);
            one(fb, 1, gxa + 1);
#pragma unroll
            for (int i = 0; i < 9; ++i) fv.set(i, F2(fa[i], fb[i]));
        },
        [&](int k) {
            const float2 v = PFLBM_LD(reinterpret_cast<const float2*>(a.sprev), k / 2, a.plane / 2);
            return F2(v.x, v.y);
        },
        [](F2, F2, F2, F2) {});
}

// L2 prefetch of the rows that the tile (pf_dx, pf_dy) tiles later in launch
// order reads, as in the one-node kernel: the population planes, g_0 (16-bit
// storage: its own int32 array), the u.grad(phi) history and, for a tile
// with walls, the node bytes. A row segment of the 64-node tile is 128 B per
// 16-bit plane and 256 B per 32-bit one; one prefetch per 128 B line. Rows
// start on a 128 B line (x0 a multiple of 64, the pitch a multiple of 64
// elements); every address lies inside the lattice's arrays.
template <int PREC>
__device__ __forceinline__ void prefetch2_l2(const StepArgs<PREC>& a, int bx, int by)
{
    const int ntx = gridDim.x, nty = gridDim.y;
    int px = bx + a.pf_dx, py = by + a.pf_dy;
    if (px >= ntx) { px -= ntx; ++py; }
    if (py >= nty) return;
    const int ntx32 = tiles_x(a.nx);
    const bool walls = a.tiles[py * ntx32 + 2 * px] == 0 || (2 * px + 1 < ntx32 && a.tiles[py * ntx32 + 2 * px + 1] == 0);
    constexpr bool F32 = PREC == PFLBM_FP32;
    // lines per row: populations (FP32: 18 planes x 2 lines; 16-bit: 17 planes
    // x 1 line and g_0 x 2), history 2, node bytes 1
    constexpr int NPOP = F32 ? 36 : 19, NL = NPOP + 3;
    for (int s = threadIdx.y * QTX + threadIdx.x; s < NL * QY; s += QTX * QY) {
        const int q = s / QY, gy = py * QY + (s - q * QY);
        if (gy >= a.ny) continue;
        const int row = gy * a.pitch + px * QX;
        const char* p;
        if (q < NPOP) {
            if (F32) {
                p = reinterpret_cast<const char*>(a.in.f + ((q >> 1) * a.plane + row)) + (q & 1) * 128;
            } else if (q < 17) {
                const int pl = q < 9 ? q : q + 1;     // plane 9 is unused: g_0 has its own array
                p = reinterpret_cast<const char*>(a.in.f + (pl * a.plane + row));
            } else {
                p = reinterpret_cast<const char*>(a.in.g0 + row) + (q - 17) * 128;
            }
        } else if (q < NPOP + 2) {
            if (a.dgdt) continue;
            p = reinterpret_cast<const char*>(a.sprev + row) + (q - NPOP) * 128;
        } else {
            if (!walls) continue;
            p = reinterpret_cast<const char*>(a.cls + row);
        }
        asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
    }
}

template <int PREC, int VV>
__global__ void __launch_bounds__(QTX * QY, PREC == PFLBM_FP32 ? PFLBM_STEP2_MINB32 : PFLBM_STEP2_MINB) k_step2(const __grid_constant__ StepArgs<PREC> a)
{
    __shared__ uint8_t s_cls[QY + 6][QCW];
    __shared__ __align__(16) float s_phi[QY + 4][QPW];
    if (PFLBM_L2_AHEAD2 > 0) prefetch2_l2<PREC>(a, blockIdx.x, blockIdx.y);
    const int x0 = blockIdx.x * QX;
    // every x the tile touches (class tile: three out) inside the lattice
    if (x0 >= 3 && x0 + QX + 3 <= a.nx)
        tile2<PREC, VV, false, PFLBM_PAIR_EARLY_F != 0>(a, blockIdx.x, blockIdx.y, s_cls, s_phi);
    else
        tile2<PREC, VV, true, PFLBM_PAIR_EARLY_F != 0>(a, blockIdx.x, blockIdx.y, s_cls, s_phi);
}

// Persistent two-node step over many lattices: work item w = (lattice,
// first 64 x 8 tile); an item covers `group` tiles of one tile column, top to
// bottom. CTAs take items w = blockIdx.x, blockIdx.x + gridDim.x, ... The
// item's lattice descriptor is copied to shared memory and read from there.
template <int PREC>
__global__ void __launch_bounds__(QTX * QY, PREC == PFLBM_FP32 ? PFLBM_STEP2_MINB32 : PFLBM_STEP2_MINB)
    k_step2_batch(const StepArgs<PREC>* __restrict__ args, const int2* __restrict__ work, int n_work, int group)
{
    __shared__ uint8_t s_cls[QY + 6][QCW];
    __shared__ __align__(16) float s_phi[QY + 4][QPW];
    __shared__ __align__(16) unsigned char s_args_raw[sizeof(StepArgs<PREC>)];
    const StepArgs<PREC>& a = *reinterpret_cast<const StepArgs<PREC>*>(s_args_raw);
    const int tid = threadIdx.y * QTX + threadIdx.x;
    for (int w = blockIdx.x; w < n_work; w += gridDim.x) {
        const int2 it = work[w];
        {
            const int* src = reinterpret_cast<const int*>(args + it.x);
            int* dst = reinterpret_cast<int*>(s_args_raw);
            for (int i = tid; i < (int)(sizeof(StepArgs<PREC>) / sizeof(int)); i += QTX * QY) dst[i] = src[i];
        }
        __syncthreads();
        const int ntx = (a.nx + QX - 1) / QX, nty = (a.ny + QY - 1) / QY;
        const int bx = it.y % ntx, by0 = it.y / ntx;
        for (int gi = 0; gi < group && by0 + gi < nty; ++gi) {
            const int x0 = bx * QX;
            if (x0 >= 3 && x0 + QX + 3 <= a.nx)
                tile2<PREC, 2, false, false>(a, bx, by0 + gi, s_cls, s_phi);
            else
                tile2<PREC, 2, true, false>(a, bx, by0 + gi, s_cls, s_phi);
            __syncthreads();   // the next tile reuses the shared tiles and descriptor
        }
    }
}

template <int PREC>
cudaError_t run2(pflbm_t* h)
{
    StepArgs<PREC> a;
    write_step_args(h, 0, &a);
    dim3 b(QTX, QY), g((h->nx + QX - 1) / QX, (h->ny + QY - 1) / QY);
    a.pf_dx = PFLBM_L2_AHEAD2 % (int)g.x;
    a.pf_dy = PFLBM_L2_AHEAD2 / (int)g.x;
    if (a.varvisc)
        k_step2<PREC, 1><<<g, b, 0, h->stream>>>(a);
    else
        k_step2<PREC, 0><<<g, b, 0, h->stream>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_step2_batch(int precision, const void* d_args, const int2* d_work, int n_work, int group,
                               int grid, cudaStream_t stream)
{
    dim3 b(QTX, QY);
    switch (precision) {
        case PFLBM_FP32:
            k_step2_batch<PFLBM_FP32><<<grid, b, 0, stream>>>((const StepArgs<PFLBM_FP32>*)d_args, d_work, n_work, group);
            break;
        case PFLBM_BF16:
            k_step2_batch<PFLBM_BF16><<<grid, b, 0, stream>>>((const StepArgs<PFLBM_BF16>*)d_args, d_work, n_work, group);
            break;
        case PFLBM_FP16:
            k_step2_batch<PFLBM_FP16><<<grid, b, 0, stream>>>((const StepArgs<PFLBM_FP16>*)d_args, d_work, n_work, group);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

int step2_batch_ctas_per_sm(int precision)
{
    int n = 0;
    cudaError_t e;
    switch (precision) {
        case PFLBM_FP32: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step2_batch<PFLBM_FP32>, QTX * QY, 0); break;
        case PFLBM_BF16: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step2_batch<PFLBM_BF16>, QTX * QY, 0); break;
        case PFLBM_FP16: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step2_batch<PFLBM_FP16>, QTX * QY, 0); break;
        default: return 1;
    }
    return e == cudaSuccess ? n : 1;
}

cudaError_t launch_step2(pflbm_t* h)
{
    switch (h->precision) {
        case PFLBM_FP32: return run2<PFLBM_FP32>(h);
        case PFLBM_BF16: return run2<PFLBM_BF16>(h);
        case PFLBM_FP16: return run2<PFLBM_FP16>(h);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pfk
