// step2.cu -- the time step with two x-adjacent nodes per thread, in packed
// FP32x2 arithmetic (FP32 and 16-bit storage), for one lattice (k_step2) and
// for groups of same-size lattices in one launch (k_step2_class).
//
// A CTA of 32 x 8 threads takes a 64 x 8 tile: thread (tx, ty) owns the
// nodes x0 + 2 tx and x0 + 2 tx + 1 of row y0 + ty. The per-node arithmetic
// is node_core (step_core.cuh) on F2 lanes: every operation of the two nodes
// is one packed instruction (add/sub/mul/fma.rn on .f32x2), each lane
// rounding exactly as the scalar code, so the results equal the one-node
// kernel's bit for bit. The pulled populations are held as raw 16-bit pairs
// (16-bit storage) and converted where used. The two nodes' values leave as
// one 32-bit (16-bit storage) or 64-bit (FP32) store per plane.
//
// All-fluid tiles: phi on a ring of one, no checks; on tiles away from the
// periodic seam the pulls of the directions without an x component are one
// aligned load for both nodes. Tiles with walls: each node's 16-bit word
// (node byte and the zeta bits of its 8 neighbours, geometry.cu) selects its
// bounce-back sources and gives a ghost node's neighbour mean, so no class
// tile is loaded; the tile's flags (k_tile2_flags) say whether phi is needed
// two nodes out and whether the tile has a zeta = 1 node at all.
//
// Each CTA first prefetches into L2 the tile that a CTA PFLBM_L2_AHEAD2
// later in launch order reads: by tensor-map box prefetches from one thread
// (k_step2, and k_step2_class in FP32), else one line prefetch per thread.
#include "step_core.cuh"

#include <cstring>
#include <type_traits>

namespace pfk {
namespace {

constexpr int QX = 64, QY = 8;        // tile (nodes)
constexpr int QTX = QX / 2;           // threads in x
constexpr int QCW = QX + 6;           // row width of a class tile for the shared pulls (never read here)
constexpr int QPW = QX + 4;           // phi tile row (halo 2)

// all-fluid tiles: pull f with g, before the phi-tile barrier (twice the
// loads in flight per thread, for 9 more registers)
#ifndef PFLBM_PAIR_EARLY_F
#define PFLBM_PAIR_EARLY_F 1
#endif

// resident 256-thread CTAs per SM asked of the kernels: 4 with 16-bit storage
// (64 registers, the pulled populations held as raw pairs), 3 with FP32
#ifndef PFLBM_STEP2_MINB
#define PFLBM_STEP2_MINB 4
#endif
#ifndef PFLBM_STEP2_MINB32
#define PFLBM_STEP2_MINB32 3
#endif

// L2 prefetch distance in CTAs of launch order (0: off): about a quarter of
// the 4 x 152 resident CTAs (distances of 76 to 228 measured within 1 %)
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
            // even element (pair indices here and below are non-negative
            // element indices halved by a shift, which a signed division by
            // two would have to sign-correct)
            if constexpr (PREC == PFLBM_FP32) {
                const float2 v = PFLBM_LD(reinterpret_cast<const float2*>(base), idx >> 1, 9LL * plane / 2);
                return F2(v.x, v.y);
            } else {
                const uint32_t u = PFLBM_LD(reinterpret_cast<const uint32_t*>(base), idx >> 1, 9LL * plane / 2);
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
            return PFLBM_LD(reinterpret_cast<const uint32_t*>(base), idx >> 1, 9LL * plane / 2);
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
        const int2 r = PFLBM_LD(reinterpret_cast<const int2*>(P.g0), (gy * pitch + gx) >> 1, plane / 2);
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

// The one-node ring around an all-fluid 64 x 8 tile: phi of one node each,
// for the first 148 threads. Called after the pair's own pulls are issued
// and before their phi is summed, so that the ring's loads are in flight
// together with the pair's (measured 0.7 to 1.4 % faster than after).
template <int PREC, bool WRAP>
__device__ __forceinline__ void ring2f(const StepArgs<PREC>& a, float (*s_phi)[QPW], int x0, int y0, int tid, bool tiny)
{
    constexpr int RW = QX + 2, NR = 2 * RW + 2 * QY;
    static_assert(NR <= QTX * QY, "one ring node per thread at most");
    if (tid < NR) {
        const int t = tid;
        int py, px;
        if (t < RW) { py = 1; px = 1 + t; }
        else if (t < 2 * RW) { py = QY + 2; px = 1 + t - RW; }
        else if (t < 2 * RW + QY) { py = 2 + t - 2 * RW; px = 1; }
        else { py = 2 + t - 2 * RW - QY; px = QX + 2; }
        const int gy = y0 - 2 + py, xr = x0 - 2 + px;
        const int gx = !WRAP ? xr : (tiny ? wrapn(xr, a.nx) : wrap1(xr, a.nx));
        s_phi[py][px] = pulled_phi<PREC, false, WRAP, QCW>(a.in, nullptr, 0, 0, gx, gy, a.nx, a.pitch, a.plane);
    }
}

// Pull of direction I at node (gx, gy) from its zeta-neighbour bits zm (bit
// j - 1: zeta(x + c_j)): streaming from x - c_I when that node is a zeta = 1
// node, else f*_{I'} of x + c_I when that one is, else the node's own
// f*_{I'} (modified bounce-back, Sec. 2.2.2). The same selection as the
// class-tile pull (step_core.cuh), one load whatever the lanes select.
template <int I, int PREC, bool WRAP>
__device__ __forceinline__ float pullm(const typename Store<PREC>::S* __restrict__ base, unsigned zm, int gx, int gy,
                                       int nx, int pitch, int plane)
{
    using T = Store<PREC>;
    constexpr int X = cx(I), Y = cy(I), O = opp(I);
    static_assert(T::template unit<I>() == T::template unit<O>(), "opposite directions share a unit");
    int src;
    if constexpr (!WRAP) {
        const int k = gy * pitch + gx;
        src = k + O * plane;
        if (zm & (1u << (I - 1))) src = k + (O * plane + Y * pitch + X);
        if (zm & (1u << (O - 1))) src = k + (I * plane - Y * pitch - X);
    } else {
        src = O * plane + gy * pitch + gx;
        if (zm & (1u << (I - 1))) src = O * plane + (gy + Y) * pitch + wrap1(gx + X, nx);
        if (zm & (1u << (O - 1))) src = I * plane + (gy - Y) * pitch + wrap1(gx - X, nx);
    }
    return T::template ldp<I>(PFLBM_LD(base, src, 9LL * plane));
}

template <int PREC, bool WRAP>
__device__ __forceinline__ void pull_fm(float v[9], const typename Store<PREC>::S* __restrict__ f, unsigned zm, int gx,
                                        int gy, int nx, int pitch, int plane)
{
    using T = Store<PREC>;
    v[0] = T::template ldp<0>(PFLBM_LD(f, gy * pitch + gx, 9LL * plane));
    v[1] = pullm<1, PREC, WRAP>(f, zm, gx, gy, nx, pitch, plane);
    v[2] = pullm<2, PREC, WRAP>(f, zm, gx, gy, nx, pitch, plane);
    v[3] = pullm<3, PREC, WRAP>(f, zm, gx, gy, nx, pitch, plane);
    v[4] = pullm<4, PREC, WRAP>(f, zm, gx, gy, nx, pitch, plane);
    v[5] = pullm<5, PREC, WRAP>(f, zm, gx, gy, nx, pitch, plane);
    v[6] = pullm<6, PREC, WRAP>(f, zm, gx, gy, nx, pitch, plane);
    v[7] = pullm<7, PREC, WRAP>(f, zm, gx, gy, nx, pitch, plane);
    v[8] = pullm<8, PREC, WRAP>(f, zm, gx, gy, nx, pitch, plane);
}

// One node's pulled g (raw g_0 and g_0..g_8); returns phi.
template <int PREC, bool WRAP>
__device__ __forceinline__ float pull_gm(float v[9], int32_t& raw, const Planes<PREC>& P, unsigned zm, int gx, int gy,
                                         int nx, int pitch, int plane)
{
    using T = Store<PREC>;
    raw = PFLBM_LD(P.g0, gy * pitch + gx, plane);
    v[0] = T::g0(raw);
    v[1] = pullm<1, PREC, WRAP>(P.g, zm, gx, gy, nx, pitch, plane);
    v[2] = pullm<2, PREC, WRAP>(P.g, zm, gx, gy, nx, pitch, plane);
    v[3] = pullm<3, PREC, WRAP>(P.g, zm, gx, gy, nx, pitch, plane);
    v[4] = pullm<4, PREC, WRAP>(P.g, zm, gx, gy, nx, pitch, plane);
    v[5] = pullm<5, PREC, WRAP>(P.g, zm, gx, gy, nx, pitch, plane);
    v[6] = pullm<6, PREC, WRAP>(P.g, zm, gx, gy, nx, pitch, plane);
    v[7] = pullm<7, PREC, WRAP>(P.g, zm, gx, gy, nx, pitch, plane);
    v[8] = pullm<8, PREC, WRAP>(P.g, zm, gx, gy, nx, pitch, plane);
    return phi_of<PREC>(v);
}

// Ring positions (width H) around a tile with walls, one or two per thread:
// their lattice coordinates, and phi of the node there from its word (0 on
// nodes that are not zeta = 1 and outside the lattice).
template <int H>
struct Ring2 {
    static constexpr int RW = QX + 2 * H, NTOP = H * RW, NSIDE = H * QY, NR = 2 * NTOP + 2 * NSIDE;
    static constexpr int N = (NR + QTX * QY - 1) / (QTX * QY);
    __device__ static __forceinline__ void pos(int t, int& py, int& px)
    {
        if (t < NTOP) { py = 2 - H + t / RW; px = 2 - H + t % RW; }
        else if (t < 2 * NTOP) { const int u = t - NTOP; py = QY + 2 + u / RW; px = 2 - H + u % RW; }
        else if (t < 2 * NTOP + NSIDE) { const int u = t - 2 * NTOP; py = 2 + u / H; px = 2 - H + u % H; }
        else { const int u = t - 2 * NTOP - NSIDE; py = 2 + u / H; px = QX + 2 + u % H; }
    }
};

// phi-tile positions the ghost fill visits (the tile and one ring) and how
// many each thread takes
constexpr int QGW = QX + 2, QGP = QGW * (QY + 2), QNG = (QGP + QTX * QY - 1) / (QTX * QY);

// Prologue of a 64 x 8 tile with walls, phi needed H nodes out. Loads in
// the order their results are needed: the words of the pair, the ring
// positions and (H = 2) the ghost-fill positions; the pair's g, selected by
// its words; the ghost-fill words into shared memory; the ring's g. Then phi, one barrier, the ghost values (H = 2: the
// zeta-weighted 3 x 3 mean of Sec. 2.2.2, b = 9, or the Robin value of
// Appendix A cases 1 and 3 on flat walls), another barrier.
template <int PREC, bool WRAP, int H>
__device__ __forceinline__ void wall_prologue(const StepArgs<PREC>& a, float (*s_phi)[QPW], uint16_t* s_gw, int x0,
                                              int y0, Hold2<PREC>& g, int32_t raw[2], uint8_t code[2], unsigned zm[2])
{
    using RG = Ring2<H>;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * QTX + tx;
    const int nx = a.nx, ny = a.ny, pitch = a.pitch;
    const bool tiny = nx < QX + 8;
    auto wx = [&](int x) { return !WRAP ? x : (tiny ? wrapn(x, nx) : wrap1(x, nx)); };
    const int gxa = x0 + 2 * tx, gy = y0 + ty;

    // words: the pair, the ring positions, the ghost-fill positions
    uint16_t w[2] = {CLS_OUT, CLS_OUT};
    if (gy < ny) {
        if (!WRAP) {
            const uint32_t wp = PFLBM_LD(reinterpret_cast<const uint32_t*>(a.nword), (gy * pitch + gxa) >> 1, a.plane / 2);
            w[0] = (uint16_t)(wp & 0xffffu);
            w[1] = (uint16_t)(wp >> 16);
        } else {
            w[0] = PFLBM_LD(a.nword, gy * pitch + wx(gxa), a.plane);
            w[1] = PFLBM_LD(a.nword, gy * pitch + wx(gxa + 1), a.plane);
        }
    }
    uint16_t rw[RG::N];
#pragma unroll
    for (int q = 0; q < RG::N; ++q) {
        rw[q] = CLS_OUT;
        const int t = tid + q * QTX * QY;
        if (t < RG::NR) {
            int py, px;
            RG::pos(t, py, px);
            const int yy = y0 - 2 + py;
            if (yy >= 0 && yy < ny) rw[q] = PFLBM_LD(a.nword, yy * pitch + wx(x0 - 2 + px), a.plane);
        }
    }
    uint16_t gw[QNG];
#pragma unroll
    for (int q = 0; q < QNG; ++q) {
        gw[q] = CLS_OUT;
        const int p = tid + q * QTX * QY;
        if (H == 2 && p < QGP) {
            const int yy = y0 - 1 + p / QGW;
            if (yy >= 0 && yy < ny) gw[q] = PFLBM_LD(a.nword, yy * pitch + wx(x0 - 1 + p % QGW), a.plane);
        }
    }

    // the pair's own pulls
    float ga[9], gb[9];
    float pha = 0.0f, phb = 0.0f;
#pragma unroll
    for (int i = 0; i < 9; ++i) ga[i] = gb[i] = 0.0f;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        code[j] = (uint8_t)(w[j] & 0xffu);
        zm[j] = w[j] >> 8;
    }
    if (gy < ny && zeta_of(code[0])) pha = pull_gm<PREC, WRAP>(ga, raw[0], a.in, zm[0], wx(gxa), gy, nx, pitch, a.plane);
    if (gy < ny && zeta_of(code[1])) phb = pull_gm<PREC, WRAP>(gb, raw[1], a.in, zm[1], wx(gxa + 1), gy, nx, pitch, a.plane);
    if (H == 2) {
#pragma unroll
        for (int q = 0; q < QNG; ++q) {
            const int p = tid + q * QTX * QY;
            if (p < QGP) s_gw[p] = gw[q];
        }
    }
    // the ring's pulls
#pragma unroll
    for (int q = 0; q < RG::N; ++q) {
        const int t = tid + q * QTX * QY;
        if (t >= RG::NR) break;
        int py, px;
        RG::pos(t, py, px);
        float ph = 0.0f;
        if (zeta_of((uint8_t)(rw[q] & 0xffu))) {
            float v[9];
            int32_t r;
            ph = pull_gm<PREC, WRAP>(v, r, a.in, rw[q] >> 8, wx(x0 - 2 + px), y0 - 2 + py, nx, pitch, a.plane);
        }
        s_phi[py][px] = ph;
    }
#pragma unroll
    for (int i = 1; i < 9; ++i) g.set(i, F2(ga[i], gb[i]));
    s_phi[ty + 2][2 * tx + 2] = pha;
    s_phi[ty + 2][2 * tx + 3] = phb;
    __syncthreads();
    if (H == 2) {
        // ghost values; the mean reads only zeta = 1 neighbours, which no
        // thread writes here
        for (int p = tid; p < QGP; p += QTX * QY) {
            const uint16_t wd = s_gw[p];
            const uint8_t c = (uint8_t)(wd & 0xffu);
            if (c == CLS_OUT || (c & CLS_MASK) != CLS_GHOST) continue;
            const int py = p / QGW + 1, px = p % QGW + 1;
            if (c & (F_GHOST_UP | F_GHOST_DOWN)) {
                const float pb = s_phi[(c & F_GHOST_UP) ? py + 1 : py - 1][px];
                s_phi[py][px] = robin_ghost<float>(pb, PFLBM_LD(a.wet, (y0 - 2 + py) * pitch + wx(x0 - 2 + px), a.plane));
                continue;
            }
            const unsigned m = wd >> 8;
            float num = 0.0f, den = 0.0f;
#pragma unroll
            for (int j = 1; j < 9; ++j) {
                if (m & (1u << (j - 1))) {
                    num += s_phi[py + cy(j)][px + cx(j)];
                    den += 1.0f;
                }
            }
            s_phi[py][px] = num / den;
        }
        __syncthreads();
    }
}

// KIND: 0 reads the tile's flags; 1 a tile known to be all fluid (the wall
// path is not compiled in); 2 a tile known to have walls. EARLY_F: on an
// all-fluid tile, pull f with g, before the phi-tile barrier.
template <int PREC, int VV, bool WRAP, bool EARLY_F, int KIND = 0>
__device__ __forceinline__ void tile2(const StepArgs<PREC>& a, int bx, int by, float (*s_phi)[QPW], uint16_t* s_gw)
{
    using T = Store<PREC>;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * QTX + tx;
    const int x0 = bx * QX, y0 = by * QY;
    const int nx = a.nx, ny = a.ny, pitch = a.pitch;
    // bit 0: both 32 x 8 halves all fluid; bit 1: phi needed two nodes out;
    // bit 2: a zeta = 1 node
    const uint8_t tflags = KIND == 1 ? (uint8_t)5 : a.tiles2[by * ((nx + QX - 1) / QX) + bx];
    if (!(tflags & 4)) return;   // no zeta = 1 node: nothing to store (the whole CTA leaves)
    const bool fluid = KIND == 1 || (KIND == 0 && (tflags & 1));
    const bool tiny = nx < QX + 8;
    const int gxa = x0 + 2 * tx, gy = y0 + ty;
    Hold2<PREC> g;
    int32_t raw[2] = {0, 0};
    uint8_t code[2] = {CLS_FLUID, CLS_FLUID};
    unsigned zm[2] = {0xffu, 0xffu};
    Hold2<PREC> fearly;

    if (fluid) {
        // ---- prologue of an all-fluid tile: no node words, no checks ----
        pull2_g<PREC, WRAP>(g, raw, a.in, gxa, gy, nx, pitch, a.plane);
        if (EARLY_F) pull2_f<PREC, WRAP>(fearly, a.in.f, gxa, gy, nx, pitch, a.plane);
        ring2f<PREC, WRAP>(a, s_phi, x0, y0, tid, tiny);
        const F2 ph = phi2<PREC>(g, raw);
        s_phi[ty + 2][2 * tx + 2] = ph.x;
        s_phi[ty + 2][2 * tx + 3] = ph.y;
        __syncthreads();
    } else {
        // ---- tile with walls: each node's word gives its class and its
        // bounce-back sources; every load is issued before the barrier ----
        if (tflags & 2)
            wall_prologue<PREC, WRAP, 2>(a, s_phi, s_gw, x0, y0, g, raw, code, zm);
        else
            wall_prologue<PREC, WRAP, 1>(a, s_phi, s_gw, x0, y0, g, raw, code, zm);
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
        const float2 l = row[(px >> 1) - 1], m = row[px >> 1], rr = row[(px >> 1) + 1];
        Wr[r] = F2(l.y, m.x);
        Cr[r] = F2(m.x, m.y);
        Er[r] = F2(m.y, rr.x);
    }
    F2 gpx, gpy, lap;
    stencil9<F2>(Cr[1], Er[1], Wr[1], Cr[2], Cr[0], Er[2], Wr[2], Wr[0], Er[0], gpx, gpy, lap);
    node_core<PREC, true, VV>(
        a, lane, Cr[1], gpx, gpy, lap, g,
        [&](Hold2<PREC>& fv) {
            if (fluid && EARLY_F) {
                fv = fearly;
            } else if (fluid) {
                pull2_f<PREC, WRAP>(fv, a.in.f, gxa, gy, nx, pitch, a.plane);
            } else {
                float fa[9], fb[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) fa[i] = fb[i] = 0.0f;
                if (lane.valid[0]) pull_fm<PREC, WRAP>(fa, a.in.f, zm[0], gxa, gy, nx, pitch, a.plane);
                if (lane.valid[1]) pull_fm<PREC, WRAP>(fb, a.in.f, zm[1], gxa + 1, gy, nx, pitch, a.plane);
#pragma unroll
                for (int i = 0; i < 9; ++i) fv.set(i, F2(fa[i], fb[i]));
            }
        },
        [&](int k) {
            const float2 v = PFLBM_LD(reinterpret_cast<const float2*>(a.sprev), k >> 1, a.plane / 2);
            return F2(v.x, v.y);
        },
        [](F2, F2, F2, F2) {});
}

// L2 prefetch by tensor-map boxes (cp.async.bulk.prefetch.tensor): one
// instruction per array and tile, issued by one thread, with no completion
// to wait for. x is a multiple of 64 elements, so every box starts on a
// 16-byte boundary.
__device__ __forceinline__ void pf_box3(const void* map, int x, int y, int z)
{
    asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];" ::"l"(map), "r"(x), "r"(y),
                 "r"(z)
                 : "memory");
}
__device__ __forceinline__ void pf_box2(const void* map, int x, int y)
{
    asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(map), "r"(x), "r"(y)
                 : "memory");
}

// L2 prefetch of the rows that the tile (pf_dx, pf_dy) tiles later in launch
// order reads, as in the one-node kernel: the population planes, g_0 (16-bit
// storage: its own int32 array), the u.grad(phi) history and, for a tile
// with walls, the node words. A row segment of the 64-node tile is 128 B per
// 16-bit plane and 256 B per 32-bit one; one prefetch per 128 B line. Rows
// start on a 128 B line (x0 a multiple of 64, the pitch a multiple of 64
// elements); every address lies inside the lattice's arrays.
//
// MAPS: when the handle has its tensor maps, one thread issues a box
// prefetch per array instead (f, g, g_0, the history and, for a tile with
// walls, the node words). Measured on the 4096 x 2048 workload: BF16 61.9k ->
// 66.6k MLUPS, FP32 42.9k -> 44.3k; the 176 line prefetches and their index
// arithmetic were about 3 % of the kernel's instructions.
template <int PREC, bool MAPS>
__device__ __forceinline__ void prefetch2_rows(const StepArgs<PREC>& a, int px, int py, int tid)
{
    constexpr bool F32 = PREC == PFLBM_FP32;
    if (MAPS && a.tma) {
        if (tid != 0) return;
        const PfMaps* m = reinterpret_cast<const PfMaps*>(a.tma + kPfMapsAt) + a.in_copy;
        const int x = px * QX, y = py * QY;
        pf_box3(m->pop, x, y, 0);
        if (F32) {
            pf_box3(m->pop, x, y, 9);
        } else {
            pf_box3(m->g16, x, y, 10);   // g_1..g_8 (plane 9 is unused: g_0 has its own array)
            pf_box2(m->g0, x, y);
        }
        if (!a.dgdt) pf_box2(m->hist, x, y);
        if ((a.tiles2[py * ((a.nx + QX - 1) / QX) + px] & 1) == 0) pf_box2(m->nword, x, y);
        return;
    }
    const bool walls = (a.tiles2[py * ((a.nx + QX - 1) / QX) + px] & 1) == 0;
    // lines per row: populations (FP32: 18 planes x 2 lines; 16-bit: 17 planes
    // x 1 line and g_0 x 2), history 2, node words 1
    constexpr int NPOP = F32 ? 36 : 19, NL = NPOP + 3;
    for (int s = tid; s < NL * QY; s += QTX * QY) {
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
            p = reinterpret_cast<const char*>(a.nword + row);
        }
        asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
    }
}

template <int PREC>
__device__ __forceinline__ void prefetch2_l2(const StepArgs<PREC>& a, int bx, int by)
{
    const int ntx = gridDim.x, nty = gridDim.y;
    int px = bx + a.pf_dx, py = by + a.pf_dy;
    if (px >= ntx) { px -= ntx; ++py; }
    if (py >= nty) return;
    prefetch2_rows<PREC, true>(a, px, py, threadIdx.y * QTX + threadIdx.x);
}

template <int PREC, int VV>
__global__ void __launch_bounds__(QTX * QY, PREC == PFLBM_FP32 ? PFLBM_STEP2_MINB32 : PFLBM_STEP2_MINB) k_step2(const __grid_constant__ StepArgs<PREC> a)
{
    __shared__ __align__(16) float s_phi[QY + 4][QPW];
    __shared__ uint16_t s_gw[QGP];
    if (PFLBM_L2_AHEAD2 > 0) prefetch2_l2<PREC>(a, blockIdx.x, blockIdx.y);
    const int x0 = blockIdx.x * QX;
    // every x the tile touches inside the lattice (the pulls of the second
    // phi ring reach three nodes out)
    if (x0 >= 3 && x0 + QX + 3 <= a.nx)
        tile2<PREC, VV, false, PFLBM_PAIR_EARLY_F != 0>(a, blockIdx.x, blockIdx.y, s_phi, s_gw);
    else
        tile2<PREC, VV, true, PFLBM_PAIR_EARLY_F != 0>(a, blockIdx.x, blockIdx.y, s_phi, s_gw);
}

// Lattices of one size in one launch: grid (tiles of one lattice, lattices),
// the lattices' step descriptors in the kernel's parameter space (read like
// the single-lattice kernel's, through uniform indexing by blockIdx.y), and
// each CTA one 64 x 8 tile with the single-lattice tile body: the tile's
// kind read from its flags, tiles without a zeta = 1 node left at once, f
// pulled with g on all-fluid tiles, and an L2 prefetch of the tile that a
// CTA PFLBM_L2_AHEAD2 later in launch order reads.
template <int PREC>
struct ClassArgs2 {
    static constexpr int K = (30 * 1024) / (int)sizeof(StepArgs<PREC>);
    int count, ntx2, ntiles, pad;
    StepArgs<PREC> a[K];
};

template <int PREC, int VV>
__global__ void __launch_bounds__(QTX * QY, PREC == PFLBM_FP32 ? PFLBM_STEP2_MINB32 : PFLBM_STEP2_MINB)
    k_step2_class(const __grid_constant__ ClassArgs2<PREC> P)
{
    __shared__ __align__(16) float s_phi[QY + 4][QPW];
    __shared__ uint16_t s_gw[QGP];
    const StepArgs<PREC>& a = P.a[blockIdx.y];
    if (PFLBM_L2_AHEAD2 > 0) {
        const int t = blockIdx.y * P.ntiles + blockIdx.x + PFLBM_L2_AHEAD2;
        if (t < P.count * P.ntiles) {
            const int l = t / P.ntiles, tt = t - l * P.ntiles;
            // box prefetches in FP32 only: with 16-bit storage they measured
            // 2 % slower on mixes of small lattices than the line prefetches
            prefetch2_rows<PREC, PREC == PFLBM_FP32>(P.a[l], tt % P.ntx2, tt / P.ntx2,
                                                     threadIdx.y * QTX + threadIdx.x);
        }
    }
    const int bx = blockIdx.x % P.ntx2, by = blockIdx.x / P.ntx2, x0 = bx * QX;
    if (x0 >= 3 && x0 + QX + 3 <= a.nx)
        tile2<PREC, VV, false, PFLBM_PAIR_EARLY_F != 0>(a, bx, by, s_phi, s_gw);
    else
        tile2<PREC, VV, true, PFLBM_PAIR_EARLY_F != 0>(a, bx, by, s_phi, s_gw);
}

template <int PREC>
cudaError_t class2(int vv, const unsigned char* descs, int count, int nx, int ny, cudaStream_t stream)
{
    using P = ClassArgs2<PREC>;
    if (count < 1 || count > P::K) return cudaErrorInvalidValue;
    static thread_local P p;   // 30 KB: off the stack; the launch copies it
    p.count = count;
    p.ntx2 = (nx + QX - 1) / QX;
    p.ntiles = p.ntx2 * ((ny + QY - 1) / QY);
    p.pad = 0;
    std::memcpy(p.a, descs, (size_t)count * sizeof(StepArgs<PREC>));
    const dim3 g(p.ntiles, count), b(QTX, QY);
    if (vv) k_step2_class<PREC, 1><<<g, b, 0, stream>>>(p);
    else k_step2_class<PREC, 0><<<g, b, 0, stream>>>(p);
    return cudaGetLastError();
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

#ifdef PFLBM_BOUNDS
unsigned bounds_violations_step2()
{
    unsigned v = 0;
    cudaMemcpyFromSymbol(&v, g_bounds_viol, sizeof(v));
    return v;
}
#else
unsigned bounds_violations_step2() { return 0; }
#endif

int step2_class_capacity(int precision)
{
    switch (precision) {
        case PFLBM_FP32: return ClassArgs2<PFLBM_FP32>::K;
        case PFLBM_BF16: return ClassArgs2<PFLBM_BF16>::K;
        case PFLBM_FP16: return ClassArgs2<PFLBM_FP16>::K;
        default: return 0;
    }
}

cudaError_t launch_step2_class(int precision, int vv, const unsigned char* descs, int count, int nx, int ny,
                               cudaStream_t stream)
{
    switch (precision) {
        case PFLBM_FP32: return class2<PFLBM_FP32>(vv, descs, count, nx, ny, stream);
        case PFLBM_BF16: return class2<PFLBM_BF16>(vv, descs, count, nx, ny, stream);
        case PFLBM_FP16: return class2<PFLBM_FP16>(vv, descs, count, nx, ny, stream);
        default: return cudaErrorInvalidValue;
    }
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
