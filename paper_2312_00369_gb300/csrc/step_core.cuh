// step_core.cuh -- the per-node arithmetic of the time step, shared by every
// step kernel (single lattice and batched; populations pulled from global
// memory or from a shared-memory ring filled by TMA). Each kernel supplies
// the pulled populations and the phi tile; everything from there on -- the
// stencils, the chemical potential with the wetting term, the moments, both
// collisions and the stores -- is this one code, so all kernels round alike.
#pragma once

#include "storage.cuh"

#include <type_traits>

namespace pfk {

// Index-checked debug build (-DPFLBM_BOUNDS): every global and staged
// shared-memory access of the step kernels goes through PFLBM_LD / PFLBM_ST,
// which check the index against the size of the buffer it addresses; an
// index outside is counted (per translation unit, read back by
// pflbm_debug_bounds) and the access is skipped (a load returns zero). The
// normal build compiles them to the plain access.
#ifdef PFLBM_BOUNDS
static __device__ unsigned g_bounds_viol = 0;
template <typename T>
__device__ __forceinline__ T bounds_load(const T* p, long long i, long long n)
{
    if (i < 0 || i >= n) {
        atomicAdd(&g_bounds_viol, 1u);
        return T();
    }
    return p[i];
}
template <typename T, typename V>
__device__ __forceinline__ void bounds_store(T* p, long long i, long long n, V v)
{
    if (i < 0 || i >= n) {
        atomicAdd(&g_bounds_viol, 1u);
        return;
    }
    p[i] = v;
}
#define PFLBM_LD(p, i, n) ::pfk::bounds_load((p), (long long)(i), (long long)(n))
#define PFLBM_ST(p, i, n, v) ::pfk::bounds_store((p), (long long)(i), (long long)(n), (v))
#else
#define PFLBM_LD(p, i, n) ((p)[i])
#define PFLBM_ST(p, i, n, v) ((p)[i] = (v))
#endif

// Tensor maps (CUtensorMap, built on the host by cuTensorMapEncodeTiled) of
// one population copy as the staged step reads it with one tile shape.
struct alignas(64) TmaSet {
    unsigned char f[128];     // planes f_0..f_8 of [18][ny][nx]: box [W][TYT][9]
    unsigned char g[128];     // g planes: box depth 9 (FP32, from plane 9) or 8 (16-bit, from plane 10)
    unsigned char g0[128];    // 16-bit formats: the int32 g_0 plane [ny][nx], box [W0][TYT]
    unsigned char cls[128];   // node bytes [ny][nx], box [WC][TYT + 6]
};

// Tensor maps of one population copy for the two-node step's L2 prefetch of
// a later 64 x 8 tile: one box prefetch each. They follow the staged step's
// sets in the same device array (kPfMapsAt TmaSet entries in).
struct alignas(64) PfMaps {
    unsigned char pop[128];   // planes of [18][ny][nx]: box [64][8][9] (f from plane 0; FP32 g from plane 9)
    unsigned char g16[128];   // 16-bit formats: box [64][8][8], g_1..g_8 from plane 10
    unsigned char g0[128];    // 16-bit formats: the int32 g_0 plane [ny][nx], box [64][8]
    unsigned char hist[128];  // the u.grad(phi) history [ny][nx], box [64][8]
    unsigned char nword[128]; // the two-node step's node words [ny][nx], box [64][8]
};
constexpr int kPfMapsAt = 4;

__device__ __forceinline__ int wrap1(int x, int nx) { return x < 0 ? x + nx : (x >= nx ? x - nx : x); }
__device__ __forceinline__ int wrapn(int x, int nx) { int r = x % nx; return r < 0 ? r + nx : r; }

template <int PREC>
struct StepArgs {
    using T = Store<PREC>;
    using S = typename T::S;
    using C = typename T::C;
    const uint8_t* cls;
    const uint8_t* tiles;  // per tile: 1 when every node within 2 of it is fluid
    const C* wet;
    Planes<PREC> in, out;
    C* sprev;
    int nx, ny, pitch;
    int plane;      // 18 * plane < 2^31 (checked at create)
    C beta4, kappa, rho_g, drho, omega_f, omega_g, force_pre, alpha;
    C tau_g3h, dtau3;    // variable viscosity: tau_f = tau_g3h + dtau3 phi
    C gx, gy;            // body acceleration
    int varvisc;
    int dgdt;            // 0: backward difference of G (history read/written); 1: omitted
    int pf_dx, pf_dy;    // k_step L2 prefetch target: PFLBM_L2_AHEAD CTAs on, in tiles
    const TmaSet* tma;   // staged step: tensor maps [tile shape][population copy]
    const uint8_t* sflags[2];   // staged step: tile flags of each shape (fluid, ring of two)
    const uint16_t* nword;      // two-node step: node byte | zeta-neighbour bits << 8
    const uint8_t* tiles2;      // two-node step: 64 x 8 tile flags (all fluid, ring of two)
    int in_copy;         // which population copy `in` is (index into tma)
    int* status;
    // macroscopic output (read-back kernel only), dense [ny][nx]
    double* o_phi;
    double* o_u;
    double* o_p;
    // the same fields rounded to float (read-back kernel only)
    float* f_phi;
    float* f_u;
    float* f_p;
};

// Whether a node takes the bounce-back pull. Per warp: if any active lane
// has an unknown link, all take it (for a node without one it reads what
// the plain pull reads), so a warp issues one set of loads.
__device__ __forceinline__ bool has_link(uint8_t code)
{
    return __any_sync(__activemask(), (code & F_LINK) != 0);
}

template <typename C>
__device__ __forceinline__ C sum_moving(const C v[9])
{
    return ((v[1] + v[2]) + (v[3] + v[4])) + ((v[5] + v[6]) + (v[7] + v[8]));
}

// sum_{i != 0} v_i in population units (v in the step's work units).
template <int PREC>
__device__ __forceinline__ typename Store<PREC>::C sum_pop(const typename Store<PREC>::C v[9])
{
    using T = Store<PREC>;
    if constexpr (T::kNorm)
        return fmadd(T::template unit<1>(), (v[1] + v[2]) + (v[3] + v[4]),
                     T::template unit<5>() * ((v[5] + v[6]) + (v[7] + v[8])));
    else
        return sum_moving(v);
}

// phi = sum_i g_i (Eq. order-parameter), in one fixed order everywhere.
template <int PREC>
__device__ __forceinline__ typename Store<PREC>::C phi_of(const typename Store<PREC>::C v[9])
{
    return v[0] + sum_pop<PREC>(v);
}

// Ghost value of a flat wall under the Robin condition n_w . grad(phi) =
// c (phi_w - phi_w^2) with phi_w = (phi_b + phi_g) / 2 (Appendix A cases 1
// and 3): d = phi_b - phi_g solves (c/4) d^2 + (1 - c (phi_b - 1/2)) d
// - c (phi_b - phi_b^2) = 0, taken in the form that is regular at c = 0.
template <typename C>
__host__ __device__ __forceinline__ C robin_ghost(C pb, C c)
{
    const C A = c * C(0.25), B = C(1) - c * (pb - C(0.5)), Cc = c * (pb - pb * pb);
    const C d = C(2) * Cc / (B + sqrt(B * B + C(4) * A * Cc));
    return pb - d;
}

// The class tile's row width is a template argument with a default (the
// argument is not deduced from the pointer, which may be nullptr).
template <class T> struct NoDeduce { using type = T; };

// Pull of direction I at node (gx, gy), whose class byte sits at s_cls[sy][sx].
// CHECK = false: every neighbour is a zeta = 1 node (s_cls is not read).
// WRAP = false: the neighbours x +- 1 lie inside 0..nx-1 (a tile away from the
// periodic seam), so every source is the node's own index plus a fixed offset.
template <int I, int PREC, bool CHECK, bool WRAP, int CW = TX + 6>
__device__ __forceinline__ typename Store<PREC>::C pull(const typename Store<PREC>::S* __restrict__ base,
                                                        typename NoDeduce<const uint8_t (*)[CW]>::type s_cls, int sy, int sx, int gx,
                                                        int gy, int nx, int pitch, int plane)
{
    using T = Store<PREC>;
    constexpr int X = cx(I), Y = cy(I), O = opp(I);
    if constexpr (!WRAP) {
        const int k = gy * pitch + gx;
        if (!CHECK) return T::template ldp<I>(PFLBM_LD(base, k + (I * plane - Y * pitch - X), 9LL * plane));
        int src = k + O * plane;
        if (zeta_of(s_cls[sy + Y][sx + X])) src = k + (O * plane + Y * pitch + X);
        if (zeta_of(s_cls[sy - Y][sx - X])) src = k + (I * plane - Y * pitch - X);
        return T::template ldp<I>(PFLBM_LD(base, src, 9LL * plane));
    }
    if (!CHECK)
        return T::template ldp<I>(PFLBM_LD(base, I * plane + (gy - Y) * pitch + wrap1(gx - X, nx), 9LL * plane));
    // one load from the selected source, no branch (a warp whose lanes pick
    // different sources still issues one load); I and O share a storage unit
    static_assert(T::template unit<I>() == T::template unit<O>(), "opposite directions share a unit");
    int src = O * plane + gy * pitch + gx;
    if (zeta_of(s_cls[sy + Y][sx + X])) src = O * plane + (gy + Y) * pitch + wrap1(gx + X, nx);
    if (zeta_of(s_cls[sy - Y][sx - X])) src = I * plane + (gy - Y) * pitch + wrap1(gx - X, nx);
    return T::template ldp<I>(PFLBM_LD(base, src, 9LL * plane));
}

template <int PREC, bool CHECK, bool WRAP, int CW = TX + 6>
__device__ __forceinline__ void pull_f(typename Store<PREC>::C v[9], const typename Store<PREC>::S* __restrict__ f,
                                       typename NoDeduce<const uint8_t (*)[CW]>::type s_cls, int sy, int sx, int gx, int gy, int nx,
                                       int pitch, int plane)
{
    using T = Store<PREC>;
    v[0] = T::template ldp<0>(PFLBM_LD(f, gy * pitch + gx, 9LL * plane));
    v[1] = pull<1, PREC, CHECK, WRAP, CW>(f, s_cls, sy, sx, gx, gy, nx, pitch, plane);
    v[2] = pull<2, PREC, CHECK, WRAP, CW>(f, s_cls, sy, sx, gx, gy, nx, pitch, plane);
    v[3] = pull<3, PREC, CHECK, WRAP, CW>(f, s_cls, sy, sx, gx, gy, nx, pitch, plane);
    v[4] = pull<4, PREC, CHECK, WRAP, CW>(f, s_cls, sy, sx, gx, gy, nx, pitch, plane);
    v[5] = pull<5, PREC, CHECK, WRAP, CW>(f, s_cls, sy, sx, gx, gy, nx, pitch, plane);
    v[6] = pull<6, PREC, CHECK, WRAP, CW>(f, s_cls, sy, sx, gx, gy, nx, pitch, plane);
    v[7] = pull<7, PREC, CHECK, WRAP, CW>(f, s_cls, sy, sx, gx, gy, nx, pitch, plane);
    v[8] = pull<8, PREC, CHECK, WRAP, CW>(f, s_cls, sy, sx, gx, gy, nx, pitch, plane);
}

// Pulled g at a node: g_0 raw (storage form) and its value, g_1..g_8.
template <int PREC, bool CHECK, bool WRAP, int CW = TX + 6>
__device__ __forceinline__ void pull_g(typename Store<PREC>::C v[9], typename Store<PREC>::G0T& raw0,
                                       const Planes<PREC>& P, typename NoDeduce<const uint8_t (*)[CW]>::type s_cls, int sy, int sx,
                                       int gx, int gy, int nx, int pitch, int plane)
{
    using T = Store<PREC>;
    raw0 = PFLBM_LD(P.g0, gy * pitch + gx, plane);
    v[0] = T::g0(raw0);
    v[1] = pull<1, PREC, CHECK, WRAP, CW>(P.g, s_cls, sy, sx, gx, gy, nx, pitch, plane);
    v[2] = pull<2, PREC, CHECK, WRAP, CW>(P.g, s_cls, sy, sx, gx, gy, nx, pitch, plane);
    v[3] = pull<3, PREC, CHECK, WRAP, CW>(P.g, s_cls, sy, sx, gx, gy, nx, pitch, plane);
    v[4] = pull<4, PREC, CHECK, WRAP, CW>(P.g, s_cls, sy, sx, gx, gy, nx, pitch, plane);
    v[5] = pull<5, PREC, CHECK, WRAP, CW>(P.g, s_cls, sy, sx, gx, gy, nx, pitch, plane);
    v[6] = pull<6, PREC, CHECK, WRAP, CW>(P.g, s_cls, sy, sx, gx, gy, nx, pitch, plane);
    v[7] = pull<7, PREC, CHECK, WRAP, CW>(P.g, s_cls, sy, sx, gx, gy, nx, pitch, plane);
    v[8] = pull<8, PREC, CHECK, WRAP, CW>(P.g, s_cls, sy, sx, gx, gy, nx, pitch, plane);
}

template <int PREC, bool CHECK, bool WRAP, int CW = TX + 6>
__device__ __forceinline__ typename Store<PREC>::C pulled_phi(const Planes<PREC>& P, typename NoDeduce<const uint8_t (*)[CW]>::type s_cls,
                                                              int sy, int sx, int gx, int gy, int nx, int pitch,
                                                              int plane)
{
    typename Store<PREC>::C v[9];
    typename Store<PREC>::G0T raw0;
    pull_g<PREC, CHECK, WRAP, CW>(v, raw0, P, s_cls, sy, sx, gx, gy, nx, pitch, plane);
    return phi_of<PREC>(v);
}

// ---------------------------------------------------------------------------
// Lanes. The per-node arithmetic below is written once for a "lane" type C:
// the precision's scalar (one node per thread), or F2, two x-adjacent nodes
// of one thread held in a pair of registers and combined with Blackwell's
// packed FP32x2 instructions (add/sub/mul/fma.rn.f32x2: each lane is one
// IEEE operation, so a node's values are the same bit for bit as with the
// scalar code). A lane policy L supplies what differs: the node bytes,
// the wetting coefficient, the stores and the stability check.
// ---------------------------------------------------------------------------
struct F2 {
    float x, y;
    __host__ __device__ constexpr F2() : x(0.f), y(0.f) {}
    __host__ __device__ constexpr F2(float s) : x(s), y(s) {}
    __host__ __device__ constexpr F2(double s) : x((float)s), y((float)s) {}
    __host__ __device__ constexpr F2(int s) : x((float)s), y((float)s) {}
    __host__ __device__ constexpr F2(float a, float b) : x(a), y(b) {}
};
__device__ __forceinline__ float2 f2v(F2 a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ F2 v2f(float2 a) { return F2(a.x, a.y); }
// The packed operations are emitted as PTX with an explicit .rn rounding
// modifier. Even so, a packed multiply whose product fed a packed add was
// measured to come out fused into one FMA (a last-place difference from the
// scalar code, which -fmad=false keeps unfused). The per-node code below
// therefore never feeds a product into a separate add or subtract: each such
// pair is written as one fmadd, which both lane types round alike.
__device__ __forceinline__ unsigned long long f2b(F2 a)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
}
__device__ __forceinline__ F2 b2f(unsigned long long r)
{
    float x, y;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(r));
    return F2(x, y);
}
__device__ __forceinline__ F2 operator+(F2 a, F2 b)
{
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2b(a)), "l"(f2b(b)));
    return b2f(d);
}
__device__ __forceinline__ F2 operator-(F2 a, F2 b)
{
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2b(a)), "l"(f2b(b)));
    return b2f(d);
}
__device__ __forceinline__ F2 operator*(F2 a, F2 b)
{
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2b(a)), "l"(f2b(b)));
    return b2f(d);
}
__device__ __forceinline__ F2 fmadd(F2 a, F2 b, F2 c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(f2b(a)), "l"(f2b(b)), "l"(f2b(c)));
    return b2f(d);
}
__device__ __forceinline__ F2 operator-(F2 a) { return F2(-a.x, -a.y); }
__device__ __forceinline__ F2 operator/(F2 a, F2 b) { return F2(a.x / b.x, a.y / b.y); }
__device__ __forceinline__ F2& operator+=(F2& a, F2 b) { a = a + b; return a; }

// Stencils of Eqs. gradient and Laplace from the 3x3 neighbourhood.
template <typename C>
__device__ __forceinline__ void stencil9(C c, C E, C W, C N, C Sx, C NE, C NW, C SW, C SE, C& gx, C& gy, C& lap)
{
    gx = fmadd(E - W, C(1) / C(3), ((NE + SE) - (NW + SW)) * (C(1) / C(12)));
    gy = fmadd(N - Sx, C(1) / C(3), ((NE + NW) - (SE + SW)) * (C(1) / C(12)));
    lap = fmadd((E + W) + (N + Sx), C(2) / C(3), fmadd((NE + NW) + (SE + SW), C(1) / C(6), c * (C(-10) / C(3))));
}

// The same at phi-tile position (py, px).
template <typename C, int PW>
__device__ __forceinline__ void stencils(const C (*s_phi)[PW], int py, int px, C& gx, C& gy, C& lap)
{
    stencil9<C>(s_phi[py][px], s_phi[py][px + 1], s_phi[py][px - 1], s_phi[py + 1][px], s_phi[py - 1][px],
                s_phi[py + 1][px + 1], s_phi[py + 1][px - 1], s_phi[py - 1][px - 1], s_phi[py - 1][px + 1], gx, gy,
                lap);
}

// One node per thread, stored at index k.
template <int PREC>
struct Lane1 {
    using T = Store<PREC>;
    using C = typename T::C;
    using FArr = C[9];
    uint8_t code;
    int k;
    typename T::G0T g0raw;
    __device__ __forceinline__ C wet(const StepArgs<PREC>& a) const
    {
        return (code & F_WET) ? PFLBM_LD(a.wet, k, a.plane) : C(0);
    }
    __device__ __forceinline__ void check_u(const StepArgs<PREC>& a, C uu) const
    {
        if (!(uu < C(0.09))) atomicOr(a.status, 1);
    }
    template <int I>
    __device__ __forceinline__ void store_f(const StepArgs<PREC>& a, C v) const
    {
        PFLBM_ST(a.out.f, I * a.plane + k, 9LL * a.plane, T::template stp<I>(v));
    }
    // returns the storage rounding residual (computed minus stored, work units)
    template <int I>
    __device__ __forceinline__ C store_g(const StepArgs<PREC>& a, C v) const
    {
        const typename T::S s = T::template stp<I>(v);
        PFLBM_ST(a.out.g, I * a.plane + k, 9LL * a.plane, s);
        if (T::kAbsorb) return v - T::template ldp<I>(s);
        return C(0);
    }
    __device__ __forceinline__ void store_g0(const StepArgs<PREC>& a, C d) const
    {
        PFLBM_ST(a.out.g0, k, a.plane, T::g0_add(g0raw, d, a.status));
    }
    __device__ __forceinline__ void store_sprev(const StepArgs<PREC>& a, C s) const
    {
        PFLBM_ST(a.sprev, k, a.plane, s);
    }
};

// Pulled populations of two x-adjacent nodes as they are held through the
// step: F2 values (FP32 storage), or the raw 16-bit pairs (lane x in the
// low half), converted where used, which keeps them in half the registers.
template <int PREC>
struct Hold2 {
    static constexpr bool kRaw = PREC != PFLBM_FP32;
    using W = typename std::conditional<kRaw, uint32_t, F2>::type;
    W w[9];
    __device__ static __forceinline__ uint32_t pack_raw(F2 v)
    {
        if constexpr (PREC == PFLBM_BF16) {
            __nv_bfloat162 h = __float22bfloat162_rn(f2v(v));
            return *reinterpret_cast<uint32_t*>(&h);
        } else {
            __half2 h = __float22half2_rn(f2v(v));
            return *reinterpret_cast<uint32_t*>(&h);
        }
    }
    __device__ static __forceinline__ F2 unpack_raw(uint32_t u)
    {
        if constexpr (PREC == PFLBM_BF16) {
            // a BF16 value is the upper half of the FP32 value: lane x = low
            // half moved up (byte permute), lane y = high half masked
            // (measured 2 % faster in the step than the conversion intrinsic)
            uint32_t lo, hi;
            asm("prmt.b32 %0, %1, 0, 0x1044;" : "=r"(lo) : "r"(u));
            asm("and.b32 %0, %1, 0xffff0000;" : "=r"(hi) : "r"(u));
            return F2(__uint_as_float(lo), __uint_as_float(hi));
        }
        else return v2f(__half22float2(*reinterpret_cast<__half2*>(&u)));
    }
    __device__ __forceinline__ F2 operator[](int i) const
    {
        if constexpr (kRaw) return unpack_raw(w[i]);
        else return w[i];
    }
    // both lanes' values in work units (a 16-bit round trip is exact)
    __device__ __forceinline__ void set(int i, F2 v)
    {
        if constexpr (kRaw) w[i] = pack_raw(v);
        else w[i] = v;
    }
};

// Two x-adjacent nodes per thread: lane x at the even index k, lane y at
// k + 1. valid[j]: lane j is a zeta = 1 node of the lattice (stores of an
// invalid lane write values no pull reads: a zeta = 0 node, or the padding
// column nx of an odd-width lattice). FP32 and 16-bit storage.
template <int PREC>
struct Lane2 {
    using T = Store<PREC>;
    using C = F2;
    static_assert(PREC != PFLBM_FP64, "packed lanes are FP32");
    uint8_t code[2];
    bool valid[2];
    int k;
    int32_t g0raw[2];
    __device__ __forceinline__ C wet(const StepArgs<PREC>& a) const
    {
        return F2((code[0] & F_WET) ? PFLBM_LD(a.wet, k, a.plane) : 0.0f,
                  (code[1] & F_WET) ? PFLBM_LD(a.wet, k + 1, a.plane) : 0.0f);
    }
    __device__ __forceinline__ void check_u(const StepArgs<PREC>& a, C uu) const
    {
        if ((valid[0] && !(uu.x < 0.09f)) || (valid[1] && !(uu.y < 0.09f))) atomicOr(a.status, 1);
    }
    using FArr = Hold2<PREC>;
    __device__ __forceinline__ uint32_t pack(F2 v) const { return Hold2<PREC>::pack_raw(v); }
    __device__ __forceinline__ F2 unpack(uint32_t u) const { return Hold2<PREC>::unpack_raw(u); }
    template <int I>
    __device__ __forceinline__ void store_f(const StepArgs<PREC>& a, C v) const
    {
        if constexpr (PREC == PFLBM_FP32)
            PFLBM_ST(reinterpret_cast<float2*>(a.out.f), (I * a.plane + k) >> 1, 9LL * a.plane / 2, f2v(v));
        else
            PFLBM_ST(reinterpret_cast<uint32_t*>(a.out.f), (I * a.plane + k) >> 1, 9LL * a.plane / 2, pack(v));
    }
    template <int I>
    __device__ __forceinline__ C store_g(const StepArgs<PREC>& a, C v) const
    {
        if constexpr (PREC == PFLBM_FP32) {
            PFLBM_ST(reinterpret_cast<float2*>(a.out.g), (I * a.plane + k) >> 1, 9LL * a.plane / 2, f2v(v));
            return C(0);
        } else {
            const uint32_t s = pack(v);
            PFLBM_ST(reinterpret_cast<uint32_t*>(a.out.g), (I * a.plane + k) >> 1, 9LL * a.plane / 2, s);
            return v - unpack(s);
        }
    }
    // g_0 = raw + rint(d 2^30) per lane, as Fixed30::add; an overflow is
    // reported only for a valid lane
    __device__ __forceinline__ int32_t g0_lane(int32_t raw, float d, bool ok, const StepArgs<PREC>& a) const
    {
        long long q = (long long)raw + __float2ll_rn(d * 1073741824.0f);
        if (q > INT_MAX || q < -INT_MAX) {
            if (ok) atomicOr(a.status, 2);
            q = q > 0 ? INT_MAX : -INT_MAX;
        }
        return (int32_t)q;
    }
    __device__ __forceinline__ void store_g0(const StepArgs<PREC>& a, C d) const
    {
        const int2 v = make_int2(g0_lane(g0raw[0], d.x, valid[0], a), g0_lane(g0raw[1], d.y, valid[1], a));
        PFLBM_ST(reinterpret_cast<int2*>(a.out.g0), k >> 1, a.plane / 2, v);
    }
    __device__ __forceinline__ void store_sprev(const StepArgs<PREC>& a, C s) const
    {
        PFLBM_ST(reinterpret_cast<float2*>(a.sprev), k >> 1, a.plane / 2, f2v(s));
    }
};

// Collision of the opposite pair (I, O) of D2Q9. With c = c_I, f^eq (Eqs.
// feq_i, Siu) and the forcing of Eq. GGi split into a part even in c and a
// part odd in c:
//   omega f^eq_i + F_i = w (S +- A),
//   S = omega (3 p + rho (9/2 (c.u)^2 - 3/2 u.u)) + 3 (1 - 1/(2 tau)) (c.u)(c.grad rho),
//   A = 3 omega rho (c.u) + 3 (1 - 1/(2 tau)) (c.F),
// so f*_I = (1 - omega) f_I + w (S + A) and f*_O = (1 - omega) f_O + w (S - A).
// K holds the per-node constants base = omega (3 p - 3/2 rho u.u),
// c45 = 9/2 omega rho, c3 = 3 omega rho, pre3 = 3 (1 - 1/(2 tau)), omf = 1 - omega.
template <typename C>
struct PairK { C base, c45, c3, pre3, omf; };

template <int PREC, int I, int O, typename L>
__device__ __forceinline__ void collide_f_pair(const StepArgs<PREC>& a, const L& lane, typename L::C fI,
                                               typename L::C fO, const PairK<typename L::C>& K, typename L::C ux,
                                               typename L::C uy, typename L::C Fx, typename L::C Fy,
                                               typename L::C drx, typename L::C dry)
{
    using T = Store<PREC>;
    using C = typename L::C;
    static_assert(cx(O) == -cx(I) && cy(O) == -cy(I), "opposite pair");
    const C w = C(wgt<typename T::C>(I));
    const C cu = cdot<cx(I), cy(I)>(ux, uy);
    const C cF = cdot<cx(I), cy(I)>(Fx, Fy);
    const C cdr = cdot<cx(I), cy(I)>(drx, dry);
    // 16-bit work units f~ = f scale / w: the factor w becomes scale, which
    // the caller has folded into K
    const C S = fmadd(cu, fmadd(K.c45, cu, K.pre3 * cdr), K.base);
    const C A = fmadd(K.c3, cu, K.pre3 * cF);
    // w (S +- A) as fma(w, S, +-(w A)): a product never feeds a separate add
    // (the packed lanes must round as the scalar code does, and a packed
    // multiply followed by a packed add may be fused)
    C sI, sO;
    if constexpr (T::kNorm) {
        sI = S + A;
        sO = S - A;
    } else {
        const C wA = w * A;
        sI = fmadd(w, S, wA);
        sO = fmadd(w, S, -wA);
    }
    lane.template store_f<I>(a, fmadd(K.omf, fI, sI));
    lane.template store_f<O>(a, fmadd(K.omf, fO, sO));
}

// g_i (i != 0) collision and store; returns the storage rounding residual
// (population computed minus population stored) for the 16-bit formats.
template <int PREC, int I, typename L>
__device__ __forceinline__ typename L::C collide_g_dir(const StepArgs<PREC>& a, const L& lane, typename L::C g_i,
                                                       typename L::C omg, typename L::C gadd)
{
    // g*_i = (1 - omega_g) g_i + w_i (omega_g alpha mu + h_i src): gadd is the
    // second term, the same for the four axes and for the four diagonals
    return lane.template store_g<I>(a, fmadd(omg, g_i, gadd));
}

// The time step of one node (or two, in packed lanes) once its g has been
// pulled and the phi stencils are taken: chemical potential, coupling
// fields, moments, both collisions and the stores. g[i] (i = 1..8) gives the
// pulled g_i in the lane type (an array, or a Hold2). pull_f(f) fills the
// pulled f (called where the moments need it) and sprev(k) the u.grad(phi)
// history of the previous step (called only with the (1/2) dG/dt term). With
// COLLIDE = false (one lane only) readback(phi, ux, uy, p) receives the
// macroscopic fields instead. VV: 0 uniform tau_f, 1 variable viscosity,
// 2 decided by a.varvisc.
template <int PREC, bool COLLIDE, int VV, typename L, typename GA, typename PullF, typename SprevF, typename ReadF>
__device__ __forceinline__ void node_core(const StepArgs<PREC>& a, const L& lane, typename L::C ph,
                                          typename L::C gpx, typename L::C gpy, typename L::C lap,
                                          const GA& g, PullF&& pull_f, SprevF&& sprev, ReadF&& readback)
{
    using T = Store<PREC>;
    using C = typename L::C;
    using R = typename T::C;   // the scalar arithmetic type
    typename L::FArr f;

    // ---- chemical potential (Eq. chemical_potencial2) ----
    const C wet = lane.wet(a);
    const C mu = fmadd(-wet, fmadd(-ph, ph, ph),
                       fmadd(-C(a.kappa), lap, C(a.beta4) * ph * (ph - C(1)) * (ph - C(0.5))));

    // ---- coupling fields (Sec. 2.1.1): F = F_s + F_b, F_s = mu grad(phi), F_b = rho g ----
    const C rho = fmadd(C(a.drho), ph, C(a.rho_g));
    const C drx = C(a.drho) * gpx, dry = C(a.drho) * gpy;
    const C Fx = fmadd(mu, gpx, rho * C(a.gx)), Fy = fmadd(mu, gpy, rho * C(a.gy));

    // ---- hydrodynamic moments (Sec. 2.1.2) ----
    pull_f(f);
    C mx, my;
    if constexpr (T::kNorm) {
        mx = fmadd(C(T::template unit<1>()), f[1] - f[3], C(T::template unit<5>()) * ((f[5] - f[6]) + (f[8] - f[7])));
        my = fmadd(C(T::template unit<1>()), f[2] - f[4], C(T::template unit<5>()) * ((f[5] + f[6]) - (f[7] + f[8])));
    } else {
        mx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
        my = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
    }
    const C inv_rho = C(1) / rho;
    const C ux = fmadd(C(0.5), Fx, mx) * inv_rho;
    const C uy = fmadd(C(0.5), Fy, my) * inv_rho;
    const C uu = fmadd(ux, ux, uy * uy);
    C fsum;
    if constexpr (T::kNorm)
        fsum = fmadd(C(T::template unit<1>()), (f[1] + f[2]) + (f[3] + f[4]),
                     C(T::template unit<5>()) * ((f[5] + f[6]) + (f[7] + f[8])));
    else
        fsum = ((f[1] + f[2]) + (f[3] + f[4])) + ((f[5] + f[6]) + (f[7] + f[8]));
    // p = c_s^2/(1 - w_0) [sum_{i!=0} f_i + u.grad(rho)/2 + rho s_0(u)], s_0 = -w_0 (3/2) u^2
    const C p = C(0.6) * fmadd(-(rho * C(R(2) / R(3))), uu, fmadd(C(0.5), fmadd(ux, drx, uy * dry), fsum));

    if constexpr (!COLLIDE) {
        readback(ph, ux, uy, p);
        return;
    } else {
        lane.check_u(a, uu);
        // relaxation of f: uniform, or tau_f(x) = nu(phi) / c_s^2 + 1/2 with
        // nu(phi) = phi (nu_l - nu_g) + nu_g (Secs. 2.1.1, 2.1.2)
        C omega_f = C(a.omega_f), force_pre = C(a.force_pre);
        if (VV == 1 || (VV == 2 && a.varvisc)) {
            omega_f = C(1) / fmadd(C(a.dtau3), ph, C(a.tau_g3h));
            force_pre = fmadd(C(-0.5), omega_f, C(1));
        }

        // ---- f collision: f* = f + (f^eq - f)/tau_f + F_i ----
        {
            const C feq0 = fmadd(-(rho * C(wgt<R>(0) * R(1.5))), uu, C(R(-5) / R(3)) * p);
            C d0f;
            if constexpr (T::kNorm) d0f = fmadd(feq0, C(R(1) / T::template unit<0>()), -f[0]);
            else d0f = feq0 - f[0];
            lane.template store_f<0>(a, fmadd(omega_f, d0f, f[0]));
        }
        {
            PairK<C> K;
            K.base = omega_f * fmadd(-(C(1.5) * rho), uu, C(3) * p);
            K.c45 = omega_f * C(4.5) * rho;
            K.c3 = omega_f * C(3) * rho;
            K.pre3 = C(3) * force_pre;
            K.omf = C(1) - omega_f;
            if constexpr (T::kNorm) {          // scale is a power of two: exact
                K.base = K.base * C(T::scale());
                K.c45 = K.c45 * C(T::scale());
                K.c3 = K.c3 * C(T::scale());
                K.pre3 = K.pre3 * C(T::scale());
            }
            collide_f_pair<PREC, 1, 3>(a, lane, f[1], f[3], K, ux, uy, Fx, Fy, drx, dry);
            collide_f_pair<PREC, 2, 4>(a, lane, f[2], f[4], K, ux, uy, Fx, Fy, drx, dry);
            collide_f_pair<PREC, 5, 7>(a, lane, f[5], f[7], K, ux, uy, Fx, Fy, drx, dry);
            collide_f_pair<PREC, 6, 8>(a, lane, f[6], f[8], K, ux, uy, Fx, Fy, drx, dry);
        }

        // ---- g collision: g* = g + (g^eq - g)/tau_g + (3/2) G_i(t) - (1/2) G_i(t-1) ----
        const C s_now = fmadd(ux, gpx, uy * gpy);
        const C src = a.dgdt ? s_now : fmadd(C(1.5), s_now, C(-0.5) * sprev(lane.k));
        const C am = C(a.alpha) * mu;
        const C omg = C(1) - C(a.omega_g), oam = C(a.omega_g) * am;
        // h = -1/2 on the axes, 1 on the diagonals; in the 16-bit work units the
        // factor w_i is scale for every direction
        const C g_ax = C(T::kNorm ? R(T::scale()) : wgt<R>(1)) * fmadd(C(-0.5), src, oam);
        const C g_dg = C(T::kNorm ? R(T::scale()) : wgt<R>(5)) * fmadd(C(a.omega_g), am, src);
        C r_ax = collide_g_dir<PREC, 1>(a, lane, g[1], omg, g_ax);
        r_ax += collide_g_dir<PREC, 2>(a, lane, g[2], omg, g_ax);
        r_ax += collide_g_dir<PREC, 3>(a, lane, g[3], omg, g_ax);
        r_ax += collide_g_dir<PREC, 4>(a, lane, g[4], omg, g_ax);
        C r_dg = collide_g_dir<PREC, 5>(a, lane, g[5], omg, g_dg);
        r_dg += collide_g_dir<PREC, 6>(a, lane, g[6], omg, g_dg);
        r_dg += collide_g_dir<PREC, 7>(a, lane, g[7], omg, g_dg);
        r_dg += collide_g_dir<PREC, 8>(a, lane, g[8], omg, g_dg);
        // storage rounding residual in population units (0 for FP32 / FP64)
        const C resid = T::kAbsorb
                            ? fmadd(C(T::template unit<1>()), r_ax, C(T::template unit<5>()) * r_dg)
                            : C(0);
        {
            // g_0^eq - g_0 = sum_{i!=0} g_i - (1 - w_0) alpha mu (Eq. H_i); in the
            // 16-bit formats g_0 also takes back what rounding removed from g_1..g_8
            C gsum;
            if constexpr (T::kNorm)
                gsum = fmadd(C(T::template unit<1>()), (g[1] + g[2]) + (g[3] + g[4]),
                             C(T::template unit<5>()) * ((g[5] + g[6]) + (g[7] + g[8])));
            else
                gsum = ((g[1] + g[2]) + (g[3] + g[4])) + ((g[5] + g[6]) + (g[7] + g[8]));
            const C d0 = fmadd(C(a.omega_g), fmadd(-C(R(1) - wgt<R>(0)), am, gsum), C(wgt<R>(0) * R(-2)) * src);
            lane.store_g0(a, T::kAbsorb ? d0 + resid : d0);
        }
        if (!a.dgdt) lane.store_sprev(a, s_now);
    }
}

// One node per thread (scalar lane) at phi-tile position (py, px) and
// lattice coordinates (gx, gy): stencils, then node_core; zeta = 0 nodes only
// write their read-back values.
template <int PREC, bool COLLIDE, int VV, int PW, typename PullF, typename SprevF>
__device__ __forceinline__ void node_step(const StepArgs<PREC>& a, uint8_t code, const typename Store<PREC>::C (*s_phi)[PW],
                                          int py, int px, int gx, int gy, const typename Store<PREC>::C g[9],
                                          typename Store<PREC>::G0T g0raw, PullF&& pull_f, SprevF&& sprev)
{
    using T = Store<PREC>;
    using C = typename T::C;
    const int k = gy * a.pitch + gx;
    const size_t o = (size_t)gy * a.nx + gx;
    const long long no = (long long)a.nx * a.ny;
    if (!zeta_of(code)) {
        if (!COLLIDE) {
            if (a.o_phi) PFLBM_ST(a.o_phi, o, no, (double)s_phi[py][px]);
            if (a.o_u) { PFLBM_ST(a.o_u, 2 * o, 2 * no, 0.0); PFLBM_ST(a.o_u, 2 * o + 1, 2 * no, 0.0); }
            if (a.o_p) PFLBM_ST(a.o_p, o, no, 0.0);
            if (a.f_phi) PFLBM_ST(a.f_phi, o, no, (float)s_phi[py][px]);
            if (a.f_u) { PFLBM_ST(a.f_u, 2 * o, 2 * no, 0.0f); PFLBM_ST(a.f_u, 2 * o + 1, 2 * no, 0.0f); }
            if (a.f_p) PFLBM_ST(a.f_p, o, no, 0.0f);
        }
        return;
    }
    C gpx, gpy, lap;
    stencils<C, PW>(s_phi, py, px, gpx, gpy, lap);
    Lane1<PREC> lane{code, k, g0raw};
    node_core<PREC, COLLIDE, VV>(a, lane, s_phi[py][px], gpx, gpy, lap, g, pull_f, sprev,
                                 [&](C ph, C ux, C uy, C p) {
                                     if (a.o_phi) PFLBM_ST(a.o_phi, o, no, (double)ph);
                                     if (a.o_u) {
                                         PFLBM_ST(a.o_u, 2 * o, 2 * no, (double)ux);
                                         PFLBM_ST(a.o_u, 2 * o + 1, 2 * no, (double)uy);
                                     }
                                     if (a.o_p) PFLBM_ST(a.o_p, o, no, (double)p);
                                     if (a.f_phi) PFLBM_ST(a.f_phi, o, no, (float)ph);
                                     if (a.f_u) {
                                         PFLBM_ST(a.f_u, 2 * o, 2 * no, (float)ux);
                                         PFLBM_ST(a.f_u, 2 * o + 1, 2 * no, (float)uy);
                                     }
                                     if (a.f_p) PFLBM_ST(a.f_p, o, no, (float)p);
                                 });
}

// Ghost values of the phi tile (halo 2): every ghost node within one node of
// the tile takes the zeta-weighted mean of its 3x3 neighbourhood (Sec.
// 2.2.2), or the Robin value of Appendix A cases 1 and 3 on flat walls.
// cls(dy, dx) and wet_at(dy, dx) give the class byte and the wetting array
// entry of the node at (y0 + dy, x0 + dx); phi-tile position (py, px) is
// that node at dy = py - 2, dx = px - 2. Called by every thread of the CTA.
template <typename C, int TXT, int TYT, int PW, typename ClsF, typename WetF>
__device__ __forceinline__ void fill_ghosts(C (*s_phi)[PW], ClsF&& cls, WetF&& wet_at, int tid, int nthreads)
{
    for (int p = tid; p < (TYT + 2) * (TXT + 2); p += nthreads) {
        int py = p / (TXT + 2) + 1, px = p % (TXT + 2) + 1;   // phi-tile coords 1..T+2
        uint8_t c = cls(py - 2, px - 2);
        if (c == CLS_OUT || (c & CLS_MASK) != CLS_GHOST) continue;
        if (c & (F_GHOST_UP | F_GHOST_DOWN)) {
            const C pb = s_phi[(c & F_GHOST_UP) ? py + 1 : py - 1][px];
            s_phi[py][px] = robin_ghost<C>(pb, wet_at(py - 2, px - 2));
            continue;
        }
        C num = C(0), den = C(0);
#pragma unroll
        for (int j = 1; j < 9; ++j) {
            if (zeta_of(cls(py - 2 + cy(j), px - 2 + cx(j)))) {
                num += s_phi[py + cy(j)][px + cx(j)];
                den += C(1);
            }
        }
        s_phi[py][px] = num / den;
    }
}

}  // namespace pfk
