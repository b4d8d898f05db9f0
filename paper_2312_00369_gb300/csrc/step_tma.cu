// step_tma.cu -- the staged time step: population rows reach shared memory by
// TMA (cp.async.bulk.tensor with mbarrier completion) instead of per-node
// global loads.
//
// Each CTA marches down a strip of TXT x TYT tiles (a tile column of one
// lattice, or a y-range of it). The rows the strip needs live in a ring of
// NS = G + 1 stages of TYT rows each: a block (one tile) reads rows y0 - 3 ..
// y0 + TYT + 2 of the 18 population planes (G row groups), and the group the
// next block adds is loaded while the current block computes. A row is
// therefore read once per strip; only the 16-byte-aligned column halo is
// read again by the neighbouring strip (from L2). The node bytes come in a
// window of TYT + 6 rows per block.
//
// The window of a strip starts A = 16 / sizeof(element) columns left of it
// (a TMA box must start on a 16-byte boundary). Columns outside 0..nx-1 (x
// is periodic) and rows outside 0..ny-1 come back from TMA as zeros; the
// columns the tile needs there (three on each side) are copied from the
// wrapped positions with plain loads, and node bytes of rows outside the
// lattice are marked CLS_OUT.
//
// Once a block's data is in shared memory, every pull of Sec. 2.2.2's
// streaming and modified bounce-back is a shared-memory load, and the rest
// of the step is node_step (step_core.cuh), the arithmetic every kernel
// shares; results equal the global-load kernel's bit for bit.
//
// Waits on an mbarrier give up after about 2^31 clock cycles: the kernel then
// sets bit 4 of the status word (reported as PFLBM_ETIMEOUT), waits once more
// (bounded) for the copies it issued and returns.
//
// The host side here also encodes, after the staged step's tensor maps, the
// two-node step's prefetch maps (PfMaps, step_core.cuh): boxes of 64 x 8
// nodes that its CTAs prefetch into L2 with cp.async.bulk.prefetch.tensor.
#include <cuda.h>

#include <cstring>
#include <mutex>

#include "step_core.cuh"

namespace pfk {
namespace {

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase of parity `parity`; false after ~2^31 cycles.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity)
{
    if (mbar_try_wait(b, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(b, parity))
        if (clock64() - t0 > (1LL << 31)) return false;
    return true;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const void* map, int x, int y, int z, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const void* map, int x, int y, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void prefetch_map(const void* map) { asm volatile("prefetch.tensormap [%0];" ::"l"(map) : "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

constexpr int kThreads = 256;   // one node of the tile per thread, every tile shape

// resident CTAs per SM the staged kernels are compiled for (registers <=
// 65536 / (256 x this)); the shared-memory ring allows as many
template <int PREC> struct MinBlocks { static constexpr int v = PREC == PFLBM_FP32 ? 3 : 4; };
constexpr int kTimeoutBit = 4;  // status bit: a TMA wait gave up

__host__ __device__ constexpr int round128(int b) { return (b + 127) / 128 * 128; }

// Geometry of the staged data for one precision and tile shape.
template <int PREC, int TXT, int TYT>
struct Geo {
    using S = typename Store<PREC>::S;
    static_assert(TXT * TYT == kThreads, "one node per thread");
    static_assert((TYT & (TYT - 1)) == 0 && TXT % 32 == 0, "tile shape");
    static constexpr int ES = (int)sizeof(S);
    static constexpr int A = 16 / ES;                       // window offset of a population row (16 B)
    static constexpr int W = TXT + 2 * A;                   // window width
    static constexpr int G = (TYT + 6 + TYT - 1) / TYT;     // row groups a block reads
    static constexpr int NS = G + 1;                        // stages of the ring
    static constexpr int PL = TYT * W;                      // elements of one plane in one stage
    static constexpr bool kG0 = PREC == PFLBM_BF16 || PREC == PFLBM_FP16;   // g_0 in its own int32 plane
    static constexpr int GP0 = kG0 ? 10 : 9;                // first g plane the g box brings
    static constexpr int NGP = kG0 ? 8 : 9;                 // planes of the g box
    static constexpr int A0 = 4, W0 = TXT + 8;              // int32 g_0 window
    static constexpr int AC = 16, WC = TXT + 32, CR = TYT + 6;   // node-byte window of a block
    static constexpr int B_F = 9 * PL * ES, B_G = NGP * PL * ES, B_G0 = kG0 ? TYT * W0 * 4 : 0, B_C = CR * WC;
    static constexpr int STAGE = round128(18 * PL * ES);    // bytes of one population stage
    static constexpr int STAGE0 = round128(B_G0);
    static constexpr int CBUF = round128(B_C);
    static constexpr int PHI = round128((TYT + 4) * (TXT + 4) * (int)sizeof(typename Store<PREC>::C));
    // shared-memory layout: ring | g_0 ring | 2 node-byte windows | phi tile | barriers
    static constexpr int O_G0 = NS * STAGE;
    static constexpr int O_C = O_G0 + NS * STAGE0;
    static constexpr int O_PHI = O_C + 2 * CBUF;
    static constexpr int O_BAR = O_PHI + PHI;
    static constexpr int BYTES = O_BAR + 8 * NS + 16;
    static_assert((9 * PL * ES) % 128 == 0 && (GP0 * PL * ES) % 128 == 0, "TMA destinations 128-byte aligned");
    static constexpr uint32_t tx_bytes(bool with_cls) { return (uint32_t)(B_F + B_G + B_G0 + (with_cls ? B_C : 0)); }
};

// Addressing of the staged data while one block is computed.
template <int PREC, int TXT, int TYT>
struct View {
    using Gm = Geo<PREC, TXT, TYT>;
    using S = typename Store<PREC>::S;
    const S* pop;          // ring base
    const int32_t* g0;     // g_0 ring base (16-bit formats)
    const uint8_t* cls;    // this block's node-byte window
    int sb;                // ring stage of the block's first row group
    // element offset of window row d (d = -3 .. TYT + 2, relative to y0)
    __device__ __forceinline__ int rbase(int d) const
    {
        int st = sb + (d + 3) / TYT;
        if (st >= Gm::NS) st -= Gm::NS;
        return st * (Gm::STAGE / Gm::ES) + ((d + 3) % TYT) * Gm::W;
    }
    __device__ __forceinline__ int r0base(int d) const
    {
        int st = sb + (d + 3) / TYT;
        if (st >= Gm::NS) st -= Gm::NS;
        return st * (Gm::STAGE0 / 4) + ((d + 3) % TYT) * Gm::W0;
    }
    __device__ __forceinline__ uint8_t c(int d, int dx) const
    {
        return PFLBM_LD(cls, (d + 3) * Gm::WC + dx + Gm::AC, Gm::CR * Gm::WC);
    }
};

// Pulled populations of lattice P0 (0: f, 9: g) at window position (d, dx):
// streaming from x - c_i, or the modified bounce-back of Sec. 2.2.2 when
// CHECK (the same source choice as the global-load kernel's pull).
template <int PREC, int TXT, int TYT, bool CHECK, int P0>
__device__ __forceinline__ void spull(typename Store<PREC>::C v[9], const View<PREC, TXT, TYT>& V, int d, int dx)
{
    using T = Store<PREC>;
    using Gm = Geo<PREC, TXT, TYT>;
    const int rm = V.rbase(d - 1), r0 = V.rbase(d), rp = V.rbase(d + 1);
    const int c = dx + Gm::A;
    auto row = [&](int dy) { return dy < 0 ? rm : (dy > 0 ? rp : r0); };
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const int X = cx(i), Y = cy(i), O = opp(i);
        int src = row(-Y) + (P0 + i) * Gm::PL + c - X;
        if (CHECK) {
            const int srcs = src;
            src = r0 + (P0 + O) * Gm::PL + c;
            if (zeta_of(V.c(d + Y, dx + X))) src = row(Y) + (P0 + O) * Gm::PL + c + X;
            if (zeta_of(V.c(d - Y, dx - X))) src = srcs;
        }
        constexpr long long NE = (long long)Gm::NS * (Gm::STAGE / Gm::ES);   // ring elements
        switch (i) {   // the unit of direction i is a template argument of the load
            case 1: v[1] = T::template ldp<1>(PFLBM_LD(V.pop, src, NE)); break;
            case 2: v[2] = T::template ldp<2>(PFLBM_LD(V.pop, src, NE)); break;
            case 3: v[3] = T::template ldp<3>(PFLBM_LD(V.pop, src, NE)); break;
            case 4: v[4] = T::template ldp<4>(PFLBM_LD(V.pop, src, NE)); break;
            case 5: v[5] = T::template ldp<5>(PFLBM_LD(V.pop, src, NE)); break;
            case 6: v[6] = T::template ldp<6>(PFLBM_LD(V.pop, src, NE)); break;
            case 7: v[7] = T::template ldp<7>(PFLBM_LD(V.pop, src, NE)); break;
            default: v[8] = T::template ldp<8>(PFLBM_LD(V.pop, src, NE)); break;
        }
    }
    if (P0 == 0) v[0] = T::template ldp<0>(PFLBM_LD(V.pop, r0 + c, (long long)Gm::NS * (Gm::STAGE / Gm::ES)));
}

template <int PREC, int TXT, int TYT, bool CHECK>
__device__ __forceinline__ void spull_g(typename Store<PREC>::C v[9], typename Store<PREC>::G0T& raw0,
                                        const View<PREC, TXT, TYT>& V, int d, int dx)
{
    using T = Store<PREC>;
    using Gm = Geo<PREC, TXT, TYT>;
    spull<PREC, TXT, TYT, CHECK, 9>(v, V, d, dx);
    if constexpr (Gm::kG0) raw0 = PFLBM_LD(V.g0, V.r0base(d) + dx + Gm::A0, Gm::NS * (Gm::STAGE0 / 4));
    else raw0 = __float_as_int(PFLBM_LD(V.pop, V.rbase(d) + 9 * Gm::PL + dx + Gm::A, Gm::NS * (Gm::STAGE / Gm::ES)));
    v[0] = T::g0(raw0);
}

template <int PREC, int TXT, int TYT, bool CHECK>
__device__ __forceinline__ typename Store<PREC>::C sphi(const View<PREC, TXT, TYT>& V, int d, int dx)
{
    typename Store<PREC>::C v[9];
    typename Store<PREC>::G0T raw0;
    spull_g<PREC, TXT, TYT, CHECK>(v, raw0, V, d, dx);
    return phi_of<PREC>(v);
}

// Issue (one thread) the TMA loads of row group q of the strip at x0 into
// ring stage st, and with_cls: the node-byte window of block cb into buffer cbuf.
template <int PREC, int TXT, int TYT>
__device__ __forceinline__ void issue_group(const TmaSet* ts, unsigned char* smem, uint64_t* bars, int x0, int q, int st,
                                            bool with_cls, int cb, int cbuf)
{
    using Gm = Geo<PREC, TXT, TYT>;
    uint64_t* bar = bars + st;
    unsigned char* dst = smem + st * Gm::STAGE;
    mbar_expect_tx(bar, Gm::tx_bytes(with_cls));
    const int y = q * TYT - 3;
    tma_load_3d(dst, ts->f, x0 - Gm::A, y, 0, bar);                                      // f_0 .. f_8
    tma_load_3d(dst + Gm::GP0 * Gm::PL * Gm::ES, ts->g, x0 - Gm::A, y, Gm::GP0, bar);    // g planes
    if constexpr (Gm::kG0) tma_load_2d(smem + Gm::O_G0 + st * Gm::STAGE0, ts->g0, x0 - Gm::A0, y, bar);
    if (with_cls) tma_load_2d(smem + Gm::O_C + cbuf * Gm::CBUF, ts->cls, x0 - Gm::AC, cb * TYT - 3, bar);
}

// Copy, with plain loads, what TMA could not bring: for row group q (stage
// st), the columns within three of the strip's nodes that lie outside
// 0..nx-1 (taken from the wrapped positions); for the node-byte window of
// block cb (buffer cbuf, when with_cls), the same columns, and CLS_OUT for
// rows outside 0..ny-1. Called by every thread; the caller synchronises.
template <int PREC, int TXT, int TYT>
__device__ __forceinline__ void fix_group(const StepArgs<PREC>& a, unsigned char* smem, int x0, int q, int st,
                                          bool with_cls, int cb, int cbuf, int tid)
{
    using Gm = Geo<PREC, TXT, TYT>;
    using S = typename Store<PREC>::S;
    const int nx = a.nx, ny = a.ny;
    const int nreal = min(TXT, nx - x0);
    const bool left = x0 == 0, right = x0 + TXT >= nx;
    if (with_cls) {
        uint8_t* cw = smem + Gm::O_C + cbuf * Gm::CBUF;
        for (int p = tid; p < Gm::CR * Gm::WC; p += kThreads) {
            const int r = p / Gm::WC, y = cb * TYT - 3 + r;
            if (y < 0 || y >= ny) cw[p] = CLS_OUT;
        }
        if (left || right) {
            // 3 columns each side, CR rows
            for (int p = tid; p < 6 * Gm::CR; p += kThreads) {
                const int r = p / 6, j = p % 6, y = cb * TYT - 3 + r;
                const int dx = j < 3 ? j - 3 : nreal + (j - 3);
                if (y < 0 || y >= ny || !((j < 3 && left) || (j >= 3 && right))) continue;
                int xs = (x0 + dx) % nx;
                if (xs < 0) xs += nx;
                PFLBM_ST(cw, r * Gm::WC + dx + Gm::AC, Gm::CR * Gm::WC, PFLBM_LD(a.cls, (size_t)y * a.pitch + xs, a.plane));
            }
        }
    }
    if (!(left || right)) return;
    S* pop = reinterpret_cast<S*>(smem + st * Gm::STAGE);
    int32_t* g0r = reinterpret_cast<int32_t*>(smem + Gm::O_G0 + st * Gm::STAGE0);
    constexpr int NPL = 9 + Gm::NGP + (Gm::kG0 ? 1 : 0);   // planes to copy
    for (int p = tid; p < 6 * TYT * NPL; p += kThreads) {
        const int j = p % 6, r = (p / 6) % TYT, pl = p / (6 * TYT);
        const int y = q * TYT - 3 + r;
        const int dx = j < 3 ? j - 3 : nreal + (j - 3);
        if (y < 0 || y >= ny || !((j < 3 && left) || (j >= 3 && right))) continue;
        int xs = (x0 + dx) % nx;
        if (xs < 0) xs += nx;
        const size_t k = (size_t)y * a.pitch + xs;
        if (pl < 9) {
            PFLBM_ST(pop, pl * Gm::PL + r * Gm::W + dx + Gm::A, 18 * Gm::PL,
                     PFLBM_LD(a.in.f, (size_t)pl * a.plane + k, 18LL * a.plane));
        } else if (pl < 9 + Gm::NGP) {
            const int gp = Gm::GP0 + (pl - 9);   // plane index in the [18] layout
            PFLBM_ST(pop, gp * Gm::PL + r * Gm::W + dx + Gm::A, 18 * Gm::PL,
                     PFLBM_LD(a.in.f, (size_t)gp * a.plane + k, 18LL * a.plane));
        } else {
            PFLBM_ST(g0r, r * Gm::W0 + dx + Gm::A0, TYT * Gm::W0, (int32_t)PFLBM_LD(a.in.g0, k, a.plane));
        }
    }
}

// Ring positions (width H) around the tile: phi from the pulled g.
template <int PREC, int TXT, int TYT, int H>
__device__ __forceinline__ void sring_phi(const View<PREC, TXT, TYT>& V, typename Store<PREC>::C (*s_phi)[TXT + 4],
                                          int tid, bool fluid)
{
    using C = typename Store<PREC>::C;
    constexpr int RW = TXT + 2 * H, NTOP = H * RW, NSIDE = H * TYT, NR = 2 * NTOP + 2 * NSIDE;
    for (int t0 = 0; t0 < NR; t0 += kThreads) {
        const int t = t0 + tid;
        if (t >= NR) break;
        int py, px;
        if (t < NTOP) { py = 2 - H + t / RW; px = 2 - H + t % RW; }
        else if (t < 2 * NTOP) { const int u = t - NTOP; py = TYT + 2 + u / RW; px = 2 - H + u % RW; }
        else if (t < 2 * NTOP + NSIDE) { const int u = t - 2 * NTOP; py = 2 + u / H; px = 2 - H + u % H; }
        else { const int u = t - 2 * NTOP - NSIDE; py = 2 + u / H; px = TXT + 2 + u % H; }
        const int d = py - 2, dx = px - 2;
        C ph = C(0);
        if (fluid) {
            ph = sphi<PREC, TXT, TYT, false>(V, d, dx);
        } else {
            const uint8_t c = V.c(d, dx);
            if (zeta_of(c)) {
                if (has_link(c)) ph = sphi<PREC, TXT, TYT, true>(V, d, dx);
                else ph = sphi<PREC, TXT, TYT, false>(V, d, dx);
            }
        }
        s_phi[py][px] = ph;
    }
}

// The blocks b0 .. b0 + nb - 1 of the strip at tile column sx of one lattice.
// Row group q goes to ring stage (q - b0) % NS and block b0 + i reads
// node-byte buffer i & 1. ph holds the parity of the next phase of each
// stage's barrier (bit k for stage k); it carries over from one call to the
// next, where the tile shape (and so NS) may differ. Every group issued is
// waited for before return. Returns false after a timeout (groups may then
// still be in flight: *pending says which stages).
template <int PREC, int TXT, int TYT, int VV>
__device__ __forceinline__ bool march(const StepArgs<PREC>& a, const TmaSet* ts, const uint8_t* flags, int nsx,
                                      unsigned char* smem, uint64_t* bars, int sx, int b0, int nb, unsigned& ph,
                                      unsigned* pending)
{
    using Gm = Geo<PREC, TXT, TYT>;
    using T = Store<PREC>;
    using C = typename T::C;
    const int tid = threadIdx.x;
    const int tx = tid % TXT, ty = tid / TXT;
    const int x0 = sx * TXT;
    C(*s_phi)[TXT + 4] = reinterpret_cast<C(*)[TXT + 4]>(smem + Gm::O_PHI);
    const unsigned n0 = 0, m0 = 0;   // running indices of group b0 and block b0
    // group q has running index n0 + q - b0; block b0 + i uses node-byte buffer (m0 + i) & 1
    unsigned pend = 0;               // stages with a group in flight
    auto wait_stage = [&](int st) {
        const bool r = mbar_wait(bars + st, (ph >> st) & 1);
        if (r) {
            ph ^= 1u << st;
            pend &= ~(1u << st);
        }
        return r;
    };

    // prologue: groups b0 .. b0 + G - 1, the last with block b0's node bytes,
    // and (nb > 1) group b0 + G with block b0 + 1's
    if (tid == 0) {
        fence_proxy_async();
        for (int j = 0; j < Gm::G; ++j)
            issue_group<PREC, TXT, TYT>(ts, smem, bars, x0, b0 + j, (int)((n0 + j) % Gm::NS), j == Gm::G - 1, b0, m0 & 1);
        if (nb > 1)
            issue_group<PREC, TXT, TYT>(ts, smem, bars, x0, b0 + Gm::G, (int)((n0 + Gm::G) % Gm::NS), true, b0 + 1,
                                        (m0 + 1) & 1);
    }
    for (int j = 0; j < Gm::G + (nb > 1 ? 1 : 0); ++j) pend |= 1u << ((n0 + j) % Gm::NS);
    bool ok = true;
    for (int j = 0; j < Gm::G; ++j) ok &= wait_stage((int)((n0 + j) % Gm::NS));
    if (__syncthreads_or(!ok)) {
        *pending = pend;
        return false;
    }
    for (int j = 0; j < Gm::G; ++j)
        fix_group<PREC, TXT, TYT>(a, smem, x0, b0 + j, (int)((n0 + j) % Gm::NS), j == Gm::G - 1, b0, m0 & 1, tid);

    for (int bi = 0; bi < nb; ++bi) {
        const int b = b0 + bi;
        const unsigned mb = m0 + bi;
        if (bi > 0) {
            // group b + G - 1, issued one block ago, with this block's node bytes
            const unsigned g = n0 + bi + Gm::G - 1;
            ok = wait_stage((int)(g % Gm::NS));
            if (__syncthreads_or(!ok)) {
                *pending = pend;
                return false;
            }
            fix_group<PREC, TXT, TYT>(a, smem, x0, b + Gm::G - 1, (int)(g % Gm::NS), true, b, mb & 1, tid);
        }
        __syncthreads();   // data of block b complete; block b - 1 no longer read
        // prefetch group b + G (with block b + 1's node bytes) into the stage of group b - 1
        if (bi > 0 && bi + 1 < nb) {
            const int st = (int)((n0 + bi + Gm::G) % Gm::NS);
            if (tid == 0) {
                fence_proxy_async();
                issue_group<PREC, TXT, TYT>(ts, smem, bars, x0, b + Gm::G, st, true, b + 1, (mb + 1) & 1);
            }
            pend |= 1u << st;
        }

        View<PREC, TXT, TYT> V;
        V.pop = reinterpret_cast<const typename T::S*>(smem);
        V.g0 = reinterpret_cast<const int32_t*>(smem + Gm::O_G0);
        V.cls = smem + Gm::O_C + (mb & 1) * Gm::CBUF;
        V.sb = (int)((n0 + bi) % Gm::NS);
        const int y0 = b * TYT;

        // ---- phi tile: own nodes, ring of width 1 (2 next to ghosts), ghosts ----
        const int gx = x0 + tx, gy = y0 + ty;
        const bool mine = gx < a.nx && gy < a.ny;
        C sp = C(0);   // the u.grad(phi) history, loaded early
        if (mine && !a.dgdt) sp = PFLBM_LD(a.sprev, gy * a.pitch + gx, a.plane);
        const uint8_t tf = flags[b * nsx + sx];
        const bool fluid = (tf & 1) != 0;
        const int halo = (tf & 2) ? 2 : 1;
        const uint8_t own = fluid ? (uint8_t)CLS_FLUID : V.c(ty, tx);
        C g[9];
        typename T::G0T g0raw = 0;
        {
            C ph = C(0);
            if (fluid) {
                spull_g<PREC, TXT, TYT, false>(g, g0raw, V, ty, tx);
                ph = phi_of<PREC>(g);
            } else if (zeta_of(own)) {
                if (has_link(own)) spull_g<PREC, TXT, TYT, true>(g, g0raw, V, ty, tx);
                else spull_g<PREC, TXT, TYT, false>(g, g0raw, V, ty, tx);
                ph = phi_of<PREC>(g);
            }
            s_phi[ty + 2][tx + 2] = ph;
        }
        if (halo == 1) sring_phi<PREC, TXT, TYT, 1>(V, s_phi, tid, fluid);
        else sring_phi<PREC, TXT, TYT, 2>(V, s_phi, tid, fluid);
        __syncthreads();
        if (halo == 2) {
            fill_ghosts<C, TXT, TYT, TXT + 4>(
                s_phi, [&](int dy, int dxx) { return V.c(dy, dxx); },
                [&](int dy, int dxx) {
                    int xs = (x0 + dxx) % a.nx;
                    if (xs < 0) xs += a.nx;
                    return PFLBM_LD(a.wet, (y0 + dy) * a.pitch + xs, a.plane);
                },
                tid, kThreads);
            __syncthreads();
        }

        // ---- the node ----
        if (mine) {
            node_step<PREC, true, VV, TXT + 4>(
                a, own, s_phi, ty + 2, tx + 2, gx, gy, g, g0raw,
                [&](C fv[9]) {
                    if (!fluid && has_link(own)) spull<PREC, TXT, TYT, true, 0>(fv, V, ty, tx);
                    else spull<PREC, TXT, TYT, false, 0>(fv, V, ty, tx);
                },
                [&](int) { return sp; });
        }
    }
    return true;
}

// Before the CTA leaves after a timeout: wait (bounded) for the copies still
// in flight so that none lands in shared memory that another CTA may own.
__device__ __forceinline__ void drain(unsigned char* bars_base, unsigned ph, unsigned pending)
{
    uint64_t* bars = reinterpret_cast<uint64_t*>(bars_base);
    for (int k = 0; k < 8; ++k)
        if (pending & (1u << k)) (void)mbar_wait(bars + k, (ph >> k) & 1);
}

constexpr int kMaxStages = 8;

// TMA destinations must be 128-byte aligned: the dynamic shared memory is
// requested 128 bytes larger and used from the first aligned address.
__device__ __forceinline__ unsigned char* align128(unsigned char* p)
{
    return p + ((128u - (smem_u32(p) & 127u)) & 127u);
}

__device__ __forceinline__ void init_barriers(uint64_t* bars, int n)
{
    if (threadIdx.x == 0) {
        for (int k = 0; k < n; ++k) mbar_init(bars + k, 1);
        fence_mbar_init();
    }
    __syncthreads();
}

// One lattice: work item w = (strip w % nsx, chunk w / nsx) of L blocks.
template <int PREC, int TXT, int TYT, int VV>
__global__ void __launch_bounds__(kThreads, MinBlocks<PREC>::v) k_step_staged(const __grid_constant__ StepArgs<PREC> a, int shape, int L,
                                                           int n_items)
{
    using Gm = Geo<PREC, TXT, TYT>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = align128(smem_raw);
    const TmaSet* ts = a.tma + 2 * shape + a.in_copy;
    if (threadIdx.x == 0) {
        prefetch_map(ts->f);
        prefetch_map(ts->g);
        if (Gm::kG0) prefetch_map(ts->g0);
        prefetch_map(ts->cls);
    }
    init_barriers(reinterpret_cast<uint64_t*>(smem + Gm::O_BAR), Gm::NS);
    const int nsx = (a.nx + TXT - 1) / TXT, nby = (a.ny + TYT - 1) / TYT;
    unsigned ph = 0, pending = 0;
    for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
        const int sx = w % nsx, b0 = (w / nsx) * L;
        __syncthreads();   // the previous item's last block is no longer read
        if (!march<PREC, TXT, TYT, VV>(a, ts, a.sflags[shape], nsx, smem, reinterpret_cast<uint64_t*>(smem + Gm::O_BAR),
                                       sx, b0, min(L, nby - b0), ph, &pending)) {
            if (threadIdx.x == 0) {
                atomicOr(a.status, kTimeoutBit);
                drain(smem + Gm::O_BAR, ph, pending);
            }
            return;
        }
    }
}

// Many lattices: item = (lattice, strip, first block, blocks | shape << 16);
// each item runs with its own tile shape (0: 32 x 8, 1: 64 x 4).
template <int PREC>
__global__ void __launch_bounds__(kThreads, MinBlocks<PREC>::v) k_step_staged_batch(const StepArgs<PREC>* __restrict__ args,
                                                                 const int4* __restrict__ work, int n_work, int bar_off)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = align128(smem_raw);
    __shared__ __align__(16) unsigned char s_args_raw[sizeof(StepArgs<PREC>)];
    const StepArgs<PREC>& a = *reinterpret_cast<const StepArgs<PREC>*>(s_args_raw);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + bar_off);
    init_barriers(bars, kMaxStages);
    const int tid = threadIdx.x;
    unsigned ph = 0, pending = 0;
    for (int w = blockIdx.x; w < n_work; w += gridDim.x) {
        const int4 it = work[w];
        __syncthreads();   // the previous item (descriptor, shared data) is done
        {
            const int* src = reinterpret_cast<const int*>(args + it.x);
            int* dst = reinterpret_cast<int*>(s_args_raw);
            for (int i = tid; i < (int)(sizeof(StepArgs<PREC>) / sizeof(int)); i += kThreads) dst[i] = src[i];
        }
        __syncthreads();
        const int shape = it.w >> 16, nb = it.w & 0xffff;
        const TmaSet* ts = a.tma + 2 * shape + a.in_copy;
        bool ok;
        if (shape == 0)
            ok = march<PREC, 32, 8, 2>(a, ts, a.sflags[0], (a.nx + 31) / 32, smem, bars, it.y, it.z, nb, ph, &pending);
        else
            ok = march<PREC, 64, 4, 2>(a, ts, a.sflags[1], (a.nx + 63) / 64, smem, bars, it.y, it.z, nb, ph, &pending);
        if (!ok) {
            if (tid == 0) {
                atomicOr(a.status, kTimeoutBit);
                drain(smem + bar_off, ph, pending);
            }
            return;
        }
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
        else
            cudaGetLastError();
    });
    return fn;
}

template <int PREC, int TXT, int TYT>
bool encode_set(const pflbm_t* h, int copy, TmaSet* out)
{
    using Gm = Geo<PREC, TXT, TYT>;
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    const CUtensorMapDataType dt = PREC == PFLBM_FP32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : PREC == PFLBM_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                        : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    const cuuint64_t nx = (cuuint64_t)h->nx, ny = (cuuint64_t)h->ny, pitch = (cuuint64_t)h->pitch;
    const cuuint64_t plane = ny * pitch;
    const cuuint32_t one[3] = {1, 1, 1};
    auto ok = [](CUresult r) { return r == CUDA_SUCCESS; };
    std::memset(out, 0, sizeof(*out));
    {
        const cuuint64_t dims[3] = {nx, ny, 18};
        const cuuint64_t strides[2] = {pitch * Gm::ES, plane * Gm::ES};
        const cuuint32_t bf[3] = {(cuuint32_t)Gm::W, (cuuint32_t)TYT, 9};
        const cuuint32_t bg[3] = {(cuuint32_t)Gm::W, (cuuint32_t)TYT, (cuuint32_t)Gm::NGP};
        if (!ok(enc((CUtensorMap*)out->f, dt, 3, h->pop[copy], dims, strides, bf, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE)))
            return false;
        if (!ok(enc((CUtensorMap*)out->g, dt, 3, h->pop[copy], dims, strides, bg, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE)))
            return false;
    }
    if (Gm::kG0) {
        const cuuint64_t dims[2] = {nx, ny};
        const cuuint64_t strides[1] = {pitch * 4};
        const cuuint32_t box[2] = {(cuuint32_t)Gm::W0, (cuuint32_t)TYT};
        void* base = (char*)h->pop[copy] + 18 * plane * Gm::ES;
        if (!ok(enc((CUtensorMap*)out->g0, CU_TENSOR_MAP_DATA_TYPE_INT32, 2, base, dims, strides, box, one,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE)))
            return false;
    }
    {
        const cuuint64_t dims[2] = {nx, ny};
        const cuuint64_t strides[1] = {pitch};
        const cuuint32_t box[2] = {(cuuint32_t)Gm::WC, (cuuint32_t)Gm::CR};
        if (!ok(enc((CUtensorMap*)out->cls, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, h->cls, dims, strides, box, one,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE)))
            return false;
    }
    return true;
}

template <int PREC>
bool encode_pf(const pflbm_t* h, int copy, PfMaps* out)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    constexpr bool F32 = PREC == PFLBM_FP32;
    constexpr cuuint64_t ES = F32 ? 4 : 2;
    const CUtensorMapDataType dt = F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    const cuuint64_t nx = (cuuint64_t)h->nx, ny = (cuuint64_t)h->ny, pitch = (cuuint64_t)h->pitch;
    const cuuint64_t plane = ny * pitch;
    const cuuint32_t one[3] = {1, 1, 1};
    auto map = [&](void* m, CUtensorMapDataType t, cuuint32_t rank, void* base, const cuuint64_t* dims,
                   const cuuint64_t* strides, const cuuint32_t* box) {
        return enc((CUtensorMap*)m, t, rank, base, dims, strides, box, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    std::memset(out, 0, sizeof(*out));
    const cuuint64_t d3[3] = {nx, ny, 18}, s3[2] = {pitch * ES, plane * ES};
    const cuuint32_t b9[3] = {64, 8, 9}, b8[3] = {64, 8, 8}, b2[2] = {64, 8};
    const cuuint64_t d2[2] = {nx, ny};
    if (!map(out->pop, dt, 3, h->pop[copy], d3, s3, b9)) return false;
    if (!F32) {
        if (!map(out->g16, dt, 3, h->pop[copy], d3, s3, b8)) return false;
        const cuuint64_t s4[1] = {pitch * 4};
        if (!map(out->g0, CU_TENSOR_MAP_DATA_TYPE_INT32, 2, (char*)h->pop[copy] + 18 * plane * ES, d2, s4, b2))
            return false;
    }
    const cuuint64_t sh[1] = {pitch * 4}, sw[1] = {pitch * 2};
    if (!map(out->hist, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, h->sprev, d2, sh, b2)) return false;
    if (!map(out->nword, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, h->nword, d2, sw, b2)) return false;
    return true;
}

template <int PREC>
bool encode_all(const pflbm_t* h, TmaSet* host)
{
    for (int c = 0; c < 2; ++c) {
        if (!encode_set<PREC, 32, 8>(h, c, host + 0 * 2 + c)) return false;
        if (!encode_set<PREC, 64, 4>(h, c, host + 1 * 2 + c)) return false;
    }
    static_assert(kPfMapsAt == kStagedShapes * 2, "prefetch maps follow the staged sets");
    PfMaps* pf = reinterpret_cast<PfMaps*>(host + kPfMapsAt);
    for (int c = 0; c < 2; ++c)
        if (!encode_pf<PREC>(h, c, pf + c)) return false;
    return true;
}

template <int PREC, int TXT, int TYT>
int smem_bytes() { return Geo<PREC, TXT, TYT>::BYTES + 128; }

template <int PREC>
int batch_bar_off()
{
    return round128(std::max(Geo<PREC, 32, 8>::O_BAR, Geo<PREC, 64, 4>::O_BAR));
}
template <int PREC>
int batch_smem() { return batch_bar_off<PREC>() + 8 * kMaxStages + 128; }

template <int PREC, int TXT, int TYT, int VV>
cudaError_t prepare_single()
{
    cudaError_t e = cudaFuncSetAttribute(k_step_staged<PREC, TXT, TYT, VV>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes<PREC, TXT, TYT>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_step_staged<PREC, TXT, TYT, VV>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    return e;
}

template <int PREC, int TXT, int TYT, int VV>
cudaError_t run_single(pflbm_t* h, int shape, int L, int per_sm_cap)
{
    static std::once_flag once;
    static cudaError_t prep = cudaSuccess;
    static int per_sm = 0;
    std::call_once(once, [] {
        prep = prepare_single<PREC, TXT, TYT, VV>();
        if (prep == cudaSuccess)
            prep = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_staged<PREC, TXT, TYT, VV>, kThreads,
                                                                  smem_bytes<PREC, TXT, TYT>());
    });
    if (prep != cudaSuccess) return prep;
    StepArgs<PREC> a;
    write_step_args(h, 0, &a);
    const int nsx = (h->nx + TXT - 1) / TXT, nby = (h->ny + TYT - 1) / TYT;
    L = std::max(1, std::min(L, nby));
    const int n_items = nsx * ((nby + L - 1) / L);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    int ps = std::max(1, per_sm);
    if (per_sm_cap > 0) ps = std::min(ps, per_sm_cap);
    const int grid = std::max(1, std::min(n_items, ps * std::max(1, sms)));
    k_step_staged<PREC, TXT, TYT, VV><<<grid, kThreads, smem_bytes<PREC, TXT, TYT>(), h->stream>>>(a, shape, L, n_items);
    return cudaGetLastError();
}

template <int PREC, int VV>
cudaError_t run_single_shape(pflbm_t* h, int shape, int L, int cap)
{
    return shape == 0 ? run_single<PREC, 32, 8, VV>(h, 0, L, cap) : run_single<PREC, 64, 4, VV>(h, 1, L, cap);
}

template <int PREC>
cudaError_t run_batch(const void* d_args, const int4* d_work, int n_work, int grid, cudaStream_t stream)
{
    static std::once_flag once;
    static cudaError_t prep = cudaSuccess;
    std::call_once(once, [] {
        prep = cudaFuncSetAttribute(k_step_staged_batch<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    batch_smem<PREC>());
        if (prep == cudaSuccess)
            prep = cudaFuncSetAttribute(k_step_staged_batch<PREC>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                        cudaSharedmemCarveoutMaxShared);
    });
    if (prep != cudaSuccess) return prep;
    k_step_staged_batch<PREC><<<grid, kThreads, batch_smem<PREC>(), stream>>>((const StepArgs<PREC>*)d_args, d_work,
                                                                              n_work, batch_bar_off<PREC>());
    return cudaGetLastError();
}

template <int PREC>
int batch_per_sm()
{
    int n = 0;
    if (cudaFuncSetAttribute(k_step_staged_batch<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             batch_smem<PREC>()) != cudaSuccess ||
        cudaFuncSetAttribute(k_step_staged_batch<PREC>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_staged_batch<PREC>, kThreads, batch_smem<PREC>()) !=
            cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return std::max(1, n);
}

}  // namespace

size_t tma_sets_bytes() { return (size_t)kStagedShapes * 2 * sizeof(TmaSet) + 2 * sizeof(PfMaps); }

bool encode_tma_sets(const pflbm_t* h, TmaSet* host)
{
    switch (h->precision) {
        case PFLBM_FP32: return encode_all<PFLBM_FP32>(h, host);
        case PFLBM_BF16: return encode_all<PFLBM_BF16>(h, host);
        case PFLBM_FP16: return encode_all<PFLBM_FP16>(h, host);
        default: return false;
    }
}

cudaError_t launch_step_staged(pflbm_t* h, int shape, int L, int ctas_per_sm)
{
    const bool vv = h->prm.nu_l > 0 && h->prm.nu_g > 0;
    switch (h->precision) {
        case PFLBM_FP32:
            return vv ? run_single_shape<PFLBM_FP32, 1>(h, shape, L, ctas_per_sm)
                      : run_single_shape<PFLBM_FP32, 0>(h, shape, L, ctas_per_sm);
        case PFLBM_BF16:
            return vv ? run_single_shape<PFLBM_BF16, 1>(h, shape, L, ctas_per_sm)
                      : run_single_shape<PFLBM_BF16, 0>(h, shape, L, ctas_per_sm);
        case PFLBM_FP16:
            return vv ? run_single_shape<PFLBM_FP16, 1>(h, shape, L, ctas_per_sm)
                      : run_single_shape<PFLBM_FP16, 0>(h, shape, L, ctas_per_sm);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_step_staged_batch(int precision, const void* d_args, const int4* d_work, int n_work, int grid,
                                     cudaStream_t stream)
{
    switch (precision) {
        case PFLBM_FP32: return run_batch<PFLBM_FP32>(d_args, d_work, n_work, grid, stream);
        case PFLBM_BF16: return run_batch<PFLBM_BF16>(d_args, d_work, n_work, grid, stream);
        case PFLBM_FP16: return run_batch<PFLBM_FP16>(d_args, d_work, n_work, grid, stream);
        default: return cudaErrorInvalidValue;
    }
}

#ifdef PFLBM_BOUNDS
unsigned bounds_violations_tma()
{
    unsigned v = 0;
    cudaMemcpyFromSymbol(&v, g_bounds_viol, sizeof(v));
    return v;
}
#else
unsigned bounds_violations_tma() { return 0; }
#endif

int staged_batch_ctas_per_sm(int precision)
{
    switch (precision) {
        case PFLBM_FP32: return batch_per_sm<PFLBM_FP32>();
        case PFLBM_BF16: return batch_per_sm<PFLBM_BF16>();
        case PFLBM_FP16: return batch_per_sm<PFLBM_FP16>();
        default: return 1;
    }
}

}  // namespace pfk
