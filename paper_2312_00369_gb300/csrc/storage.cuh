// storage.cuh -- how the populations are stored in HBM for each precision.
//
//   PFLBM_FP64: every f_i, g_i is a double; arithmetic in FP64.
//   PFLBM_FP32: f_i and g_i (i != 0) are floats; g_0 is a 32-bit fixed-point
//               number q = g_0 2^30; arithmetic in FP32.
//   PFLBM_BF16, PFLBM_FP16: f_i and g_i (i != 0) are 16-bit values of
//               (population / w_i) * kScale, i.e. the deviation from w_i times
//               the rest equilibrium (which is 0 for both lattices: f^eq(p=0,
//               u=0) = 0, g_i^eq(mu=0) = 0 for i != 0), normalised per
//               direction; g_0 is the same 32-bit fixed point as in FP32 and
//               absorbs the rounding residual of the eight 16-bit g_i of its
//               node, so the stored sum_i g_i is exact to 2^-30 at every node;
//               arithmetic in FP32.
//
// Work units of the step (ldp / stp / unit): FP64 and FP32 work in population
// units. The 16-bit formats work in the stored units f~ = f scale / w_i, so a
// load or store is a bare conversion; unit<I>() = w_I / scale converts back to
// population units where a sum over directions needs them (phi, moments).
//
// Layout of one copy of the state, planes of ny * pitch elements:
//   FP64 / FP32: f_0..f_8, g_0..g_8 (the g_0 plane holds the g_0 storage);
//   16-bit:      f_0..f_8, g_0..g_8 (16-bit, the g_0 plane unused), then one
//                int32 plane for g_0.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <climits>

#include "pflbm_internal.cuh"

namespace pfk {

template <int PREC> struct Store;

template <> struct Store<PFLBM_FP64> {
    using S = double;
    using C = double;
    using G0T = double;
    static constexpr bool kAbsorb = false;
    static constexpr bool kNorm = false;
    template <int I> __device__ static C ldp(S v) { return v; }
    template <int I> __device__ static S stp(C v) { return v; }
    template <int I> __device__ static constexpr C unit() { return C(1); }
    __device__ static constexpr C scale() { return C(1); }
    template <int I> __device__ static C ld(S v) { return v; }
    template <int I> __device__ static S st(C v) { return v; }
    __device__ static C g0(G0T raw) { return raw; }
    __device__ static double g0_double(G0T raw) { return raw; }
    __device__ static G0T g0_add(G0T raw, C d, int*) { return raw + d; }
    __device__ static G0T g0_from_double(double v) { return v; }
};

struct Fixed30 {
    __device__ static float value(int32_t raw) { return (float)raw * (1.0f / 1073741824.0f); }
    __device__ static double value_d(int32_t raw) { return (double)raw * (1.0 / 1073741824.0); }
    __device__ static int32_t add(int32_t raw, float d, int* status)
    {
        long long q = (long long)raw + __float2ll_rn(d * 1073741824.0f);
        if (q > INT_MAX || q < -INT_MAX) {
            atomicOr(status, 2);
            q = q > 0 ? INT_MAX : -INT_MAX;
        }
        return (int32_t)q;
    }
    __device__ static int32_t from_double(double v)
    {
        double q = rint(v * 1073741824.0);
        return (int32_t)fmax(-(double)INT_MAX, fmin((double)INT_MAX, q));
    }
};

template <> struct Store<PFLBM_FP32> {
    using S = float;
    using C = float;
    using G0T = int32_t;
    static constexpr bool kAbsorb = false;
    static constexpr bool kNorm = false;
    template <int I> __device__ static C ldp(S v) { return v; }
    template <int I> __device__ static S stp(C v) { return v; }
    template <int I> __device__ static constexpr C unit() { return C(1); }
    __device__ static constexpr C scale() { return C(1); }
    template <int I> __device__ static C ld(S v) { return v; }
    template <int I> __device__ static S st(C v) { return v; }
    __device__ static C g0(G0T raw) { return Fixed30::value(raw); }
    __device__ static double g0_double(G0T raw) { return Fixed30::value_d(raw); }
    __device__ static G0T g0_add(G0T raw, C d, int* st) { return Fixed30::add(raw, d, st); }
    __device__ static G0T g0_from_double(double v) { return Fixed30::from_double(v); }
};

// 16-bit: value = population / w_i * kScale
template <typename H, int SCALE_LOG2> struct Store16 {
    using S = H;
    using C = float;
    using G0T = int32_t;
    static constexpr bool kAbsorb = true;
    static constexpr bool kNorm = true;
    template <int I> __device__ static C ldp(S v) { return to_float(v); }
    template <int I> __device__ static S stp(C v) { return from_float(v); }
    template <int I> __device__ static constexpr float unit() { return to_pop<I>(); }
    __device__ static constexpr float scale() { return (float)(1 << SCALE_LOG2); }
    template <int I> __device__ static constexpr float to_pop()
    {
        return wgt<float>(I) / (float)(1 << SCALE_LOG2);
    }
    template <int I> __device__ static constexpr float from_pop()
    {
        return (float)(1 << SCALE_LOG2) / wgt<float>(I);
    }
    template <int I> __device__ static C ld(S v) { return to_float(v) * to_pop<I>(); }
    template <int I> __device__ static S st(C v) { return from_float(v * from_pop<I>()); }
    __device__ static C g0(G0T raw) { return Fixed30::value(raw); }
    __device__ static double g0_double(G0T raw) { return Fixed30::value_d(raw); }
    __device__ static G0T g0_add(G0T raw, C d, int* st) { return Fixed30::add(raw, d, st); }
    __device__ static G0T g0_from_double(double v) { return Fixed30::from_double(v); }
    __device__ static float to_float(__nv_bfloat16 v) { return __bfloat162float(v); }
    __device__ static float to_float(__half v) { return __half2float(v); }
    __device__ static S from_float(float v);
};
template <> __device__ inline __nv_bfloat16 Store16<__nv_bfloat16, 0>::from_float(float v) { return __float2bfloat16_rn(v); }
template <> __device__ inline __half Store16<__half, 10>::from_float(float v) { return __float2half_rn(v); }

template <> struct Store<PFLBM_BF16> : Store16<__nv_bfloat16, 0> {};
template <> struct Store<PFLBM_FP16> : Store16<__half, 10> {};

// Plane pointers of one copy of the state.
template <int PREC> struct Planes {
    using S = typename Store<PREC>::S;
    using G0T = typename Store<PREC>::G0T;
    S* f;      // plane i at f + i * plane
    S* g;      // plane i (i >= 1) at g + i * plane
    G0T* g0;   // g_0 storage
    __host__ static Planes make(void* base, size_t plane)
    {
        Planes p;
        p.f = (S*)base;
        p.g = p.f + 9 * plane;
        if (PREC == PFLBM_BF16 || PREC == PFLBM_FP16)
            p.g0 = (G0T*)(p.f + 18 * plane);
        else
            p.g0 = (G0T*)p.g;
        return p;
    }
};

// Bytes of one copy of the state.
inline size_t state_copy_bytes(int precision, size_t plane)
{
    switch (precision) {
        case PFLBM_FP64: return 18 * plane * 8;
        case PFLBM_FP32: return 18 * plane * 4;
        default: return 18 * plane * 2 + plane * 4;
    }
}

}  // namespace pfk
