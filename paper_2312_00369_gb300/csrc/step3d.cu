// step3d.cu -- kernels of the three-dimensional form of the scheme (behind
// the pflbm3d_* entry points of capi3d.cu): f on D3Q19 (Eq. 3ci, w = 1/3,
// 1/18, 1/36, c_s^2 = 1/3), g on D3Q7 (the paper's matrix, w = 1/4, 1/8,
// c_s^2 = 1/4, Sec. 2.1.3), gradients, Laplacian and a_v with the D3Q19
// weights (Eqs. gradient, Laplace, avvv), the 27-neighbour ghost average of
// Sec. 2.2.2 (b = 27).
//
// A step is either three kernels -- (1) phi = sum of the pulled g on zeta = 1
// nodes, (2) ghost phi from the zeta-weighted 27-neighbour mean, (3) the
// collide-and-store of f and g (pull scheme and modified bounce-back as in
// 2D, see step.cu), which reads phi of the 18 neighbours for the stencils --
// or the single z-marching kernel k3_fused, which recomputes phi and the
// ghost values in shared memory. Both call the same collide-and-store body.
// Nodes are stored [nz][ny][pitch]; x and y are periodic, z has walls.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "pflbm3d_internal.cuh"
#include "storage.cuh"

using namespace pfk;

#ifndef PFLBM3D_STEP_MINB
#define PFLBM3D_STEP_MINB 4   // resident 256-thread CTAs per SM asked of the FP32 step kernel (64 registers)
#endif
#ifndef PFLBM3D_PHI_AHEAD
// k3_phi: L2 prefetch of the tile this many CTAs later in launch order (0:
// off). 1216 is one wave (8 resident CTAs on each of 152 SMs); measured
// optimum, with 2432 as good and 4864 already slower. The same prefetch in
// k3_step, whose tiles read eight times the bytes, slows it at every distance.
#define PFLBM3D_PHI_AHEAD 1216
#endif
#ifndef PFLBM3D_FUSED_MINB
#define PFLBM3D_FUSED_MINB 4  // the same for the fused z-marching kernel
#endif

#ifndef PFLBM3D_FUSED_STEP_FIRST
#define PFLBM3D_FUSED_STEP_FIRST 0   // order of the two halves of a fused-step iteration
#endif

namespace pfk3 {

// D3Q19: rest, +x, -x, +y, -y, +z, -z, then the 12 edges in opposite pairs
__host__ __device__ constexpr int q19x(int i)
{
    return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
         : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
}
__host__ __device__ constexpr int q19y(int i)
{
    return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
         : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0;
}
__host__ __device__ constexpr int q19z(int i)
{
    return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
         : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0;
}
__host__ __device__ constexpr int q19o(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
template <typename C> __host__ __device__ constexpr C q19w(int i)
{
    return i == 0 ? C(1) / C(3) : (i <= 6 ? C(1) / C(18) : C(1) / C(36));
}
// D3Q7 = the first seven D3Q19 velocities
template <typename C> __host__ __device__ constexpr C q7w(int i) { return i == 0 ? C(1) / C(4) : C(1) / C(8); }

__device__ __forceinline__ int wrap1(int x, int n) { return x < 0 ? x + n : (x >= n ? x - n : x); }

template <int PREC>
struct Args3 {
    using T = Store<PREC>;
    using S = typename T::S;
    using C = typename T::C;
    const uint8_t* cls;
    const C* wet;
    S* f_in;
    S* g_in;
    typename T::G0T* g0_in;
    S* f_out;
    S* g_out;
    typename T::G0T* g0_out;
    C* sprev;
    C* phi;
    int nx, ny, nz, pitch;
    int plane;        // nz * ny * pitch, 26 planes fit in int
    C beta4, kappa, rho_g, drho, omega_f, omega_g, force_pre, alpha;
    int dgdt;             // 1: the (1/2) dG/dt term omitted (no history read or written)
    int* status;
    double* o_phi;
    double* o_u;
    double* o_p;
    int pf_dx, pf_dy, pf_dz;   // k3_phi L2 prefetch target: PFLBM3D_PHI_AHEAD CTAs on, in tiles
    float* f_phi;     // the same fields rounded to float (read-back only)
    float* f_u;
    float* f_p;
};

template <int PREC>
__device__ __forceinline__ int nbr(const Args3<PREC>& a, int x, int y, int z, int dx, int dy, int dz)
{
    return ((z + dz) * a.ny + wrap1(y + dy, a.ny)) * a.pitch + wrap1(x + dx, a.nx);
}

// Pull of population I of a lattice with velocity I of D3Q19 at node k.
template <int I, int PREC>
__device__ __forceinline__ typename Store<PREC>::C pull3(const Args3<PREC>& a, const typename Store<PREC>::S* base,
                                                         int x, int y, int z, int k, bool check)
{
    using T = Store<PREC>;
    constexpr int X = q19x(I), Y = q19y(I), Z = q19z(I), O = q19o(I);
    static_assert(PREC == PFLBM_FP32 || PREC == PFLBM_FP64, "3D storage: loads are bare");
    const int src = nbr(a, x, y, z, -X, -Y, -Z);
    if (!check) return T::template ld<I>(base[I * a.plane + src]);
    // both class bytes read at once, then one load from the selected source
    const int dst = nbr(a, x, y, z, X, Y, Z);
    int at = O * a.plane + k;
    if (zeta_of(a.cls[dst])) at = O * a.plane + dst;
    if (zeta_of(a.cls[src])) at = I * a.plane + src;
    return T::template ld<I>(base[at]);
}

template <int PREC>
__device__ __forceinline__ void pull_g7(const Args3<PREC>& a, int x, int y, int z, int k, bool check,
                                        typename Store<PREC>::C v[7], typename Store<PREC>::G0T& raw0)
{
    raw0 = a.g0_in[k];
    v[0] = Store<PREC>::g0(raw0);
    v[1] = pull3<1, PREC>(a, a.g_in, x, y, z, k, check);
    v[2] = pull3<2, PREC>(a, a.g_in, x, y, z, k, check);
    v[3] = pull3<3, PREC>(a, a.g_in, x, y, z, k, check);
    v[4] = pull3<4, PREC>(a, a.g_in, x, y, z, k, check);
    v[5] = pull3<5, PREC>(a, a.g_in, x, y, z, k, check);
    v[6] = pull3<6, PREC>(a, a.g_in, x, y, z, k, check);
}

template <typename C>
__device__ __forceinline__ C sum6(const C v[7]) { return ((v[1] + v[2]) + (v[3] + v[4])) + (v[5] + v[6]); }

// L2 prefetch, for the phi pass, of the g rows and node bytes of the tile
// PFLBM3D_PHI_AHEAD CTAs later in launch order: (pf_dx, pf_dy, pf_dz) tiles
// from this one (32 x 8 at one z). Warps 0 and 1 only, one row segment per
// thread (at most 128 B, on a 128 B line: x0 is a multiple of 32, the pitch
// of 64). Every address lies inside the arrays: the tile exists, y < ny.
template <int PREC>
__device__ __forceinline__ void prefetch_phi_rows_l2(const Args3<PREC>& a)
{
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, q = tid >> 3;
    if (PREC == PFLBM_FP64 || q >= 8) return;
    int tx = blockIdx.x + a.pf_dx, ty = blockIdx.y + a.pf_dy, tz = blockIdx.z + a.pf_dz;
    if (tx >= (int)gridDim.x) { tx -= gridDim.x; ++ty; }
    if (ty >= (int)gridDim.y) { ty -= gridDim.y; ++tz; }
    const int y = ty * 8 + (tid & 7);
    if (tz >= (int)gridDim.z || y >= a.ny) return;
    const size_t row = ((size_t)tz * a.ny + y) * a.pitch + tx * 32;
    const void* p = q == 0 ? (const void*)(a.g0_in + row)
                  : q < 7 ? (const void*)(a.g_in + q * (size_t)a.plane + row) : (const void*)(a.cls + row);
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// (1) phi on zeta = 1 nodes. The node byte and the plain pull are issued
// together (one memory latency, not two); a warp with a bounce-back link
// then pulls again with the checks. Planes 0 and nz - 1 hold no zeta = 1
// node (the two outer planes of the mask are solid), so every plain pull
// here stays inside the box.
template <int PREC>
__global__ void __launch_bounds__(256) k3_phi(Args3<PREC> a)
{
    using C = typename Store<PREC>::C;
    if (PFLBM3D_PHI_AHEAD > 0) prefetch_phi_rows_l2<PREC>(a);
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y, z = blockIdx.z;
    if (x >= a.nx || y >= a.ny || z == 0 || z == a.nz - 1) return;
    const int k = (z * a.ny + y) * a.pitch + x;
    const uint8_t c = a.cls[k];
    C v[7];
    typename Store<PREC>::G0T r;
    pull_g7<PREC>(a, x, y, z, k, false, v, r);
    if (!zeta_of(c)) return;
    if (__any_sync(__activemask(), (c & F_LINK) != 0)) pull_g7<PREC>(a, x, y, z, k, (c & F_LINK) != 0, v, r);
    a.phi[k] = v[0] + sum6(v);
}

// (2) ghost phi: zeta-weighted mean of the 27-neighbourhood, over the list
// of ghost nodes (interior nodes keep phi = 0 from creation)
template <int PREC>
__global__ void __launch_bounds__(256) k3_ghost(Args3<PREC> a, const int* __restrict__ ghosts, int n_ghosts)
{
    using C = typename Store<PREC>::C;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_ghosts) return;
    const int k = ghosts[t];
    const int x = k % a.pitch, y = (k / a.pitch) % a.ny, z = k / (a.pitch * a.ny);
    C num = C(0), den = C(0);
    for (int dz = -1; dz <= 1; ++dz) {
        if (z + dz < 0 || z + dz >= a.nz) continue;
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int m = nbr(a, x, y, z, dx, dy, dz);
                if (zeta_of(a.cls[m])) { num += a.phi[m]; den += C(1); }
            }
    }
    a.phi[k] = num / den;
}

// Collision of the opposite pair (I, I + 1) of D3Q19. With c = c_I, f^eq
// (Eqs. feq_i, Siu) and the forcing of Eq. GGi split into a part even in c
// and a part odd in c:
//   omega f^eq_i + F_i = w (S +- A),
//   S = omega (3 p + rho (9/2 (c.u)^2 - 3/2 u.u)) + 3 (1 - 1/(2 tau)) (c.u)(c.grad rho),
//   A = 3 omega rho (c.u) + 3 (1 - 1/(2 tau)) (c.F),
// so f*_I = (1 - omega) f_I + w (S + A) and f*_{I+1} = (1 - omega) f_{I+1} + w (S - A).
// K holds the per-node constants: base = omega (3 p - 3/2 rho u.u),
// c45 = 9/2 omega rho, c3 = 3 omega rho, pre3 = 3 (1 - 1/(2 tau)).
template <typename C>
struct PairK { C base, c45, c3, pre3, omf; };

template <int PREC, int I>
__device__ __forceinline__ void collide_pair(const Args3<PREC>& a, typename Store<PREC>::C fI,
                                             typename Store<PREC>::C fO, const PairK<typename Store<PREC>::C>& K,
                                             const typename Store<PREC>::C u[3], const typename Store<PREC>::C F[3],
                                             const typename Store<PREC>::C dr[3], int k)
{
    using C = typename Store<PREC>::C;
    constexpr int X = q19x(I), Y = q19y(I), Z = q19z(I);
    const C w = q19w<C>(I);
    const C cu = cdot<X, Y, Z>(u[0], u[1], u[2]);
    const C cF = cdot<X, Y, Z>(F[0], F[1], F[2]);
    const C cd = cdot<X, Y, Z>(dr[0], dr[1], dr[2]);
    const C S = w * fmadd(cu, fmadd(K.c45, cu, K.pre3 * cd), K.base);
    const C A = w * fmadd(K.c3, cu, K.pre3 * cF);
    a.f_out[I * a.plane + k] = Store<PREC>::template st<I>(fmadd(K.omf, fI, S + A));
    a.f_out[(I + 1) * a.plane + k] = Store<PREC>::template st<I + 1>(fmadd(K.omf, fO, S - A));
}

// (3) the fused collide-and-store (COLLIDE) or the macroscopic read-back of
// one zeta = 1 node; CHECK = false is the branch-free pull of a node without
// bounce-back links
// phi_at(i): phi at x + c_i (i = 0: the node itself); load_g(v, raw0): the
// pulled g of the node. Both step kernels share this body, so their results
// are identical.
template <int PREC, bool COLLIDE, bool CHECK, typename PhiAt, typename LoadG>
__device__ __forceinline__ void step_node(const Args3<PREC>& a, int x, int y, int z, int k, uint8_t code,
                                          PhiAt phi_at, LoadG load_g)
{
    using T = Store<PREC>;
    using C = typename T::C;
    const bool check = CHECK && (code & F_LINK) != 0;
    // ---- stencils on phi (D3Q19 weights), chemical potential ----
    // opposite pairs: grad += 3 w c (v_I - v_O), lap += 6 w (v_I + v_O - 2 phi)
    const C ph = phi_at(0);
    C gp[3] = {C(0), C(0), C(0)}, lap = C(0);
#pragma unroll
    for (int i = 1; i < 19; i += 2) {
        const C vp = phi_at(i), vm = phi_at(i + 1);
        const C w3 = C(3) * q19w<C>(i);
        const C d = w3 * (vp - vm);
        if (q19x(i)) gp[0] = q19x(i) > 0 ? gp[0] + d : gp[0] - d;
        if (q19y(i)) gp[1] = q19y(i) > 0 ? gp[1] + d : gp[1] - d;
        if (q19z(i)) gp[2] = q19z(i) > 0 ? gp[2] + d : gp[2] - d;
        lap = fmadd(C(2) * w3, fmadd(C(-2), ph, vp + vm), lap);
    }
    const C wet = (code & F_WET) ? a.wet[k] : C(0);
    const C mu = fmadd(-wet, fmadd(-ph, ph, ph), fmadd(-a.kappa, lap, a.beta4 * ph * (ph - C(1)) * (ph - C(0.5))));
    const C rho = fmadd(a.drho, ph, a.rho_g);
    const C dr[3] = {a.drho * gp[0], a.drho * gp[1], a.drho * gp[2]};
    const C F[3] = {mu * gp[0], mu * gp[1], mu * gp[2]};
    // ---- hydrodynamics ----
    C f[19];
    f[0] = T::template ld<0>(a.f_in[k]);
    f[1] = pull3<1, PREC>(a, a.f_in, x, y, z, k, check);
    f[2] = pull3<2, PREC>(a, a.f_in, x, y, z, k, check);
    f[3] = pull3<3, PREC>(a, a.f_in, x, y, z, k, check);
    f[4] = pull3<4, PREC>(a, a.f_in, x, y, z, k, check);
    f[5] = pull3<5, PREC>(a, a.f_in, x, y, z, k, check);
    f[6] = pull3<6, PREC>(a, a.f_in, x, y, z, k, check);
    f[7] = pull3<7, PREC>(a, a.f_in, x, y, z, k, check);
    f[8] = pull3<8, PREC>(a, a.f_in, x, y, z, k, check);
    f[9] = pull3<9, PREC>(a, a.f_in, x, y, z, k, check);
    f[10] = pull3<10, PREC>(a, a.f_in, x, y, z, k, check);
    f[11] = pull3<11, PREC>(a, a.f_in, x, y, z, k, check);
    f[12] = pull3<12, PREC>(a, a.f_in, x, y, z, k, check);
    f[13] = pull3<13, PREC>(a, a.f_in, x, y, z, k, check);
    f[14] = pull3<14, PREC>(a, a.f_in, x, y, z, k, check);
    f[15] = pull3<15, PREC>(a, a.f_in, x, y, z, k, check);
    f[16] = pull3<16, PREC>(a, a.f_in, x, y, z, k, check);
    f[17] = pull3<17, PREC>(a, a.f_in, x, y, z, k, check);
    f[18] = pull3<18, PREC>(a, a.f_in, x, y, z, k, check);
    // the g pull and the history with the f pulls (one memory round trip,
    // not one after the f stores); the g collision then precedes the f one
    C g[7];
    typename T::G0T raw0;
    load_g(g, raw0);
    const C sp = (COLLIDE && !a.dgdt) ? a.sprev[k] : C(0);
    C m[3] = {C(0), C(0), C(0)}, fsum = C(0);
#pragma unroll
    for (int i = 1; i < 19; i += 2) {
        const C d = f[i] - f[i + 1];
        if (q19x(i)) m[0] = q19x(i) > 0 ? m[0] + d : m[0] - d;
        if (q19y(i)) m[1] = q19y(i) > 0 ? m[1] + d : m[1] - d;
        if (q19z(i)) m[2] = q19z(i) > 0 ? m[2] + d : m[2] - d;
        fsum += f[i] + f[i + 1];
    }
    const C ir = C(1) / rho;
    const C u[3] = {fmadd(C(0.5), F[0], m[0]) * ir, fmadd(C(0.5), F[1], m[1]) * ir, fmadd(C(0.5), F[2], m[2]) * ir};
    const C uu = fmadd(u[2], u[2], fmadd(u[1], u[1], u[0] * u[0]));
    // p = c_s^2/(1 - w_0) [...] = (1/2) [sum_{i!=0} f_i + u.grad(rho)/2 + rho s_0], s_0 = -uu/2
    const C udr = fmadd(u[2], dr[2], fmadd(u[1], dr[1], u[0] * dr[0]));
    const C p = C(0.5) * fmadd(-(C(0.5) * rho), uu, fmadd(C(0.5), udr, fsum));
    if (!COLLIDE) {
        const size_t o = ((size_t)z * a.ny + y) * a.nx + x;
        if (a.o_phi) a.o_phi[o] = (double)ph;
        if (a.o_u) { a.o_u[3 * o] = u[0]; a.o_u[3 * o + 1] = u[1]; a.o_u[3 * o + 2] = u[2]; }
        if (a.o_p) a.o_p[o] = (double)p;
        if (a.f_phi) a.f_phi[o] = (float)ph;
        if (a.f_u) { a.f_u[3 * o] = (float)u[0]; a.f_u[3 * o + 1] = (float)u[1]; a.f_u[3 * o + 2] = (float)u[2]; }
        if (a.f_p) a.f_p[o] = (float)p;
        return;
    }
    if (!(uu < C(0.09))) atomicOr(a.status, 1);
    // ---- phase lattice (D3Q7): G_i = w_i h_i (3/2 s - 1/2 s_prev), h_0 = -5/2, h_i = -1/2 ----
    auto collide_g = [&](const C (&g)[7], typename T::G0T raw0, C sp) {
        const C s_now = fmadd(u[2], gp[2], fmadd(u[1], gp[1], u[0] * gp[0]));
        const C src = a.dgdt ? s_now : fmadd(C(1.5), s_now, C(-0.5) * sp);
        const C am = a.alpha * mu;
        // g*_i = (1 - omega_g) g_i + w_i (omega_g alpha mu - src / 2), the same for i = 1..6
        const C gm = q7w<C>(1) * fmadd(C(-0.5), src, a.omega_g * am), omg = C(1) - a.omega_g;
#pragma unroll
        for (int i = 1; i < 7; ++i) a.g_out[i * a.plane + k] = T::template st<1>(fmadd(omg, g[i], gm));
        const C d0 = fmadd(a.omega_g, fmadd(C(-0.75), am, sum6(g)), (q7w<C>(0) * C(-2.5)) * src);
        a.g0_out[k] = T::g0_add(raw0, d0, a.status);
        if (!a.dgdt) a.sprev[k] = s_now;
    };
    collide_g(g, raw0, sp);
    a.f_out[k] = T::template st<0>(fmadd(a.omega_f, fmadd(-(C(0.5) * rho), uu, C(-2) * p) - f[0], f[0]));
    PairK<C> K;
    K.base = a.omega_f * fmadd(-(C(1.5) * rho), uu, C(3) * p);
    K.c45 = a.omega_f * C(4.5) * rho;
    K.c3 = a.omega_f * C(3) * rho;
    K.pre3 = C(3) * a.force_pre;
    K.omf = C(1) - a.omega_f;
    collide_pair<PREC, 1>(a, f[1], f[2], K, u, F, dr, k);
    collide_pair<PREC, 3>(a, f[3], f[4], K, u, F, dr, k);
    collide_pair<PREC, 5>(a, f[5], f[6], K, u, F, dr, k);
    collide_pair<PREC, 7>(a, f[7], f[8], K, u, F, dr, k);
    collide_pair<PREC, 9>(a, f[9], f[10], K, u, F, dr, k);
    collide_pair<PREC, 11>(a, f[11], f[12], K, u, F, dr, k);
    collide_pair<PREC, 13>(a, f[13], f[14], K, u, F, dr, k);
    collide_pair<PREC, 15>(a, f[15], f[16], K, u, F, dr, k);
    collide_pair<PREC, 17>(a, f[17], f[18], K, u, F, dr, k);
}

template <int PREC, bool COLLIDE>
__global__ void __launch_bounds__(256, PREC == PFLBM_FP64 ? 1 : PFLBM3D_STEP_MINB) k3_step(Args3<PREC> a)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y, z = blockIdx.z;
    if (x >= a.nx || y >= a.ny) return;
    const int k = (z * a.ny + y) * a.pitch + x;
    const uint8_t code = a.cls[k];
    if (!zeta_of(code)) {
        if (!COLLIDE) {
            const size_t o = ((size_t)z * a.ny + y) * a.nx + x;
            if (a.o_phi) a.o_phi[o] = (double)a.phi[k];
            if (a.o_u) { a.o_u[3 * o] = 0.0; a.o_u[3 * o + 1] = 0.0; a.o_u[3 * o + 2] = 0.0; }
            if (a.o_p) a.o_p[o] = 0.0;
            if (a.f_phi) a.f_phi[o] = (float)a.phi[k];
            if (a.f_u) { a.f_u[3 * o] = 0.0f; a.f_u[3 * o + 1] = 0.0f; a.f_u[3 * o + 2] = 0.0f; }
            if (a.f_p) a.f_p[o] = 0.0f;
        }
        return;
    }
    auto phi_at = [&](int i) {
        return i == 0 ? a.phi[k] : a.phi[nbr(a, x, y, z, q19x(i), q19y(i), q19z(i))];
    };
    if (__any_sync(__activemask(), (code & F_LINK) != 0))
        step_node<PREC, COLLIDE, true>(a, x, y, z, k, code, phi_at,
                                       [&](typename Store<PREC>::C (&v)[7], typename Store<PREC>::G0T& r) {
                                           pull_g7<PREC>(a, x, y, z, k, (code & F_LINK) != 0, v, r);
                                       });
    else
        step_node<PREC, COLLIDE, false>(a, x, y, z, k, code, phi_at,
                                        [&](typename Store<PREC>::C (&v)[7], typename Store<PREC>::G0T& r) {
                                            pull_g7<PREC>(a, x, y, z, k, false, v, r);
                                        });
}

// ---------------------------------------------------------------------------
// The fused step: one CTA owns a TX x TY column of nodes and marches through
// planes [zb, zb + zc). Shared memory holds, per plane:
//   P: phi on a window with a halo of 2 in x and y (36 x 12): the pulled-g
//      sum on zeta = 1 nodes, the 27-neighbour mean on ghost nodes (filled in
//      place: it reads zeta = 1 entries only), 0 elsewhere; and the node
//      bytes. Ring of 5 planes.
//   G: the pulled g of the CTA's own nodes, kept by the thread that owns the
//      node until its collision three planes later. Ring of 4 planes.
// Iteration z: P(z + 3) and step(z) | sync | ghost fill of plane z + 2 |
// sync. The ghost fill and the 2-wide halo are only done where a ghost lies
// in the 34 x 10 window of the plane (per-tile plane flags from creation),
// and the second barrier only after a fill.
// ---------------------------------------------------------------------------
constexpr int FW2 = TX + 4, FH2 = TY + 4, FN2 = FW2 * FH2;   // 36 x 12
constexpr int FT = TX * TY;
constexpr int FRING1 = 2 * (TX + 2) + 2 * TY;                // 84 halo-1 ring nodes
constexpr int FRING2 = 2 * (TX + 4) + 2 * (TY + 2);          // 92 more for halo 2
constexpr int FP = 5;

template <int PREC>
struct FusedSmem {
    using C = typename Store<PREC>::C;
    using G0T = typename Store<PREC>::G0T;
    C P[FP][FN2];
    C G[4][6][FT];
    G0T G0[4][FT];
    int xmap[FW2];      // periodic x of window column
    int ymap[FH2];      // periodic y of window row
    uint8_t cls[FP][FN2];
};

template <int PREC>
size_t fused_smem_bytes() { return sizeof(FusedSmem<PREC>); }

__device__ __forceinline__ int pslot(int z) { return (z + FP) % FP; }   // z >= -2

// window position of ring node r (halo-1 ring first, then the halo-2 ring)
__device__ __forceinline__ int ring_pos(int r)
{
    if (r < FRING1) {
        if (r < TX + 2) return 1 * FW2 + (r + 1);
        r -= TX + 2;
        if (r < TX + 2) return (TY + 2) * FW2 + (r + 1);
        r -= TX + 2;
        if (r < TY) return (r + 2) * FW2 + 1;
        r -= TY;
        return (r + 2) * FW2 + (TX + 2);
    }
    r -= FRING1;
    if (r < TX + 4) return r;
    r -= TX + 4;
    if (r < TX + 4) return (TY + 3) * FW2 + r;
    r -= TX + 4;
    if (r < TY + 2) return (r + 1) * FW2;
    r -= TY + 2;
    return (r + 1) * FW2 + (TX + 3);
}

// phi (and, for own nodes, g) of window position w of plane zp
template <int PREC, bool OWN>
__device__ __forceinline__ void fused_phi_node(const Args3<PREC>& a, FusedSmem<PREC>& sm, int zp, int w, int t)
{
    using C = typename Store<PREC>::C;
    const int sp = pslot(zp);
    if (zp < 0 || zp >= a.nz) {
        sm.cls[sp][w] = CLS_INTERIOR;
        sm.P[sp][w] = C(0);
        return;
    }
    const int gx = sm.xmap[w % FW2], gy = sm.ymap[w / FW2];
    const int k = (zp * a.ny + gy) * a.pitch + gx;
    const uint8_t c = a.cls[k];
    sm.cls[sp][w] = c;
    if (!zeta_of(c)) {
        sm.P[sp][w] = C(0);
        return;
    }
    C v[7];
    typename Store<PREC>::G0T r;
    if (__any_sync(__activemask(), (c & F_LINK) != 0))
        pull_g7<PREC>(a, gx, gy, zp, k, (c & F_LINK) != 0, v, r);
    else
        pull_g7<PREC>(a, gx, gy, zp, k, false, v, r);
    sm.P[sp][w] = v[0] + sum6(v);
    if (OWN) {
        const int sg = zp & 3;
#pragma unroll
        for (int j = 0; j < 6; ++j) sm.G[sg][j][t] = v[j + 1];
        sm.G0[sg][t] = r;
    }
}

template <int PREC>
__device__ __forceinline__ void fused_phi_plane(const Args3<PREC>& a, FusedSmem<PREC>& sm, int zp, bool halo2)
{
    const int t = threadIdx.y * TX + threadIdx.x;
    fused_phi_node<PREC, true>(a, sm, zp, (threadIdx.y + 2) * FW2 + threadIdx.x + 2, t);
    const int nring = halo2 ? FRING1 + FRING2 : FRING1;
    for (int r = t; r < nring; r += FT) fused_phi_node<PREC, false>(a, sm, zp, ring_pos(r), t);
}

// ghost values of plane zq on the 34 x 10 window, in place
template <int PREC>
__device__ __forceinline__ void fused_fill_plane(const Args3<PREC>& a, FusedSmem<PREC>& sm, int zq)
{
    using C = typename Store<PREC>::C;
    const int sq = pslot(zq);
    for (int i = threadIdx.y * TX + threadIdx.x; i < (TX + 2) * (TY + 2); i += FT) {
        const int w = (i / (TX + 2) + 1) * FW2 + (i % (TX + 2)) + 1;
        if ((sm.cls[sq][w] & CLS_MASK) != CLS_GHOST) continue;
        // same summation order as k3_ghost
        C num = C(0), den = C(0);
        for (int dz = -1; dz <= 1; ++dz) {
            if (zq + dz < 0 || zq + dz >= a.nz) continue;
            const int s2 = pslot(zq + dz);
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int m = w + dy * FW2 + dx;
                    if (zeta_of(sm.cls[s2][m])) { num += sm.P[s2][m]; den += C(1); }
                }
        }
        sm.P[sq][w] = num / den;
    }
}

template <int PREC>
__global__ void __launch_bounds__(256, PREC == PFLBM_FP64 ? 1 : PFLBM3D_FUSED_MINB)
k3_fused(Args3<PREC> a, int zc, const uint8_t* __restrict__ gflag)
{
    using C = typename Store<PREC>::C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FusedSmem<PREC>& sm = *reinterpret_cast<FusedSmem<PREC>*>(smem_raw);
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int tiles = gridDim.x * gridDim.y, tile = blockIdx.y * gridDim.x + blockIdx.x;
    const int zb = 1 + blockIdx.z * zc, ze = min(zb + zc, a.nz - 1);   // zeta = 1 planes are 1 .. nz-2
    const int tx = threadIdx.x, ty = threadIdx.y, t = ty * TX + tx;
    const int x = x0 + tx, y = y0 + ty;
    // ghost in the 34 x 10 window of plane z (planes outside the lattice: none)
    auto ghosts_at = [&](int z) { return z >= 0 && z < a.nz && gflag[(size_t)z * tiles + tile] != 0; };
    auto halo2_at = [&](int z) { return ghosts_at(z - 1) || ghosts_at(z) || ghosts_at(z + 1); };
    if (t < FW2) sm.xmap[t] = ((x0 - 2 + t) % a.nx + a.nx) % a.nx;
    if (t < FH2) sm.ymap[t] = ((y0 - 2 + t) % a.ny + a.ny) % a.ny;
    __syncthreads();
    // warm-up: P(zb-2) .. P(zb+2), then the ghost values of zb-1 .. zb+1
    for (int zp = zb - 2; zp <= zb + 2; ++zp) fused_phi_plane<PREC>(a, sm, zp, halo2_at(zp));
    __syncthreads();
    for (int zq = zb - 1; zq <= zb + 1; ++zq)
        if (ghosts_at(zq)) fused_fill_plane<PREC>(a, sm, zq);
    __syncthreads();
    // Iteration z: step(z) and P(z + 3) in one phase (their loads overlap),
    // barrier, ghost values of plane z + 2, barrier if any were filled.
    // P(z + 3) takes slot (z - 2) mod 5, which step(z) does not read; the
    // planes in use are z - 1 .. z + 3.
    for (int z = zb; z < ze; ++z) {
        if (!PFLBM3D_FUSED_STEP_FIRST) fused_phi_plane<PREC>(a, sm, z + 3, halo2_at(z + 3));
        if (x < a.nx && y < a.ny) {
            const uint8_t code = sm.cls[pslot(z)][(ty + 2) * FW2 + tx + 2];
            if (zeta_of(code)) {
                const int k = (z * a.ny + y) * a.pitch + x;
                const int w = (ty + 2) * FW2 + tx + 2;
                auto phi_at = [&](int i) { return sm.P[pslot(z + q19z(i))][w + q19y(i) * FW2 + q19x(i)]; };
                const int sg = z & 3;
                auto load_g = [&](C (&v)[7], typename Store<PREC>::G0T& r) {
                    r = sm.G0[sg][t];
                    v[0] = Store<PREC>::g0(r);
#pragma unroll
                    for (int j = 0; j < 6; ++j) v[j + 1] = sm.G[sg][j][t];
                };
                if (__any_sync(__activemask(), (code & F_LINK) != 0))
                    step_node<PREC, true, true>(a, x, y, z, k, code, phi_at, load_g);
                else
                    step_node<PREC, true, false>(a, x, y, z, k, code, phi_at, load_g);
            }
        }
        if (PFLBM3D_FUSED_STEP_FIRST) fused_phi_plane<PREC>(a, sm, z + 3, halo2_at(z + 3));
        __syncthreads();
        if (ghosts_at(z + 2)) {
            fused_fill_plane<PREC>(a, sm, z + 2);
            __syncthreads();
        }
    }
}

// per tile and plane: 1 if a ghost node lies in the tile's 34 x 10 window
__global__ void k3_ghost_flags(const uint8_t* cls, int nx, int ny, int nz, int pitch, int tiles_x, uint8_t* gflag)
{
    const int tile = blockIdx.x, z = blockIdx.y;
    const int x0 = (tile % tiles_x) * TX, y0 = (tile / tiles_x) * TY;
    int any = 0;
    for (int i = threadIdx.x; i < (TX + 2) * (TY + 2); i += blockDim.x) {
        const int x = ((x0 - 1 + i % (TX + 2)) % nx + nx) % nx, y = ((y0 - 1 + i / (TX + 2)) % ny + ny) % ny;
        if ((cls[((size_t)z * ny + y) * pitch + x] & CLS_MASK) == CLS_GHOST) any = 1;
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) gflag[(size_t)z * gridDim.x + tile] = (uint8_t)any;
}

// ghost nodes: count, then list (any order: each ghost value depends on
// zeta = 1 nodes only)
__global__ void k3_ghost_collect(const uint8_t* cls, int nx, int ny, int nz, int pitch, int* count, int* list)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y, z = blockIdx.z;
    if (x >= nx || y >= ny) return;
    const int k = (z * ny + y) * pitch + x;
    if ((cls[k] & CLS_MASK) != CLS_GHOST) return;
    const int i = atomicAdd(count, 1);
    if (list) list[i] = k;
}

// ---- geometry: classes (D3Q19 neighbourhood), a_v = |n| / 12 with the
// integer n = sum 36 w_i c_i eps (36 w = 2 axes, 1 edges), flags ----
__global__ void k3_cls1(const uint8_t* solid, uint8_t* cls, int nx, int ny, int nz, int pitch)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y, z = blockIdx.z;
    if (x >= nx || y >= ny) return;
    const size_t k = ((size_t)z * ny + y) * pitch + x;
    if (!solid[k]) { cls[k] = CLS_FLUID; return; }
    bool touch = false;
    for (int i = 1; i < 19; ++i) {
        int zz = z + q19z(i);
        if (zz < 0 || zz >= nz) continue;
        size_t m = ((size_t)zz * ny + wrap1(y + q19y(i), ny)) * pitch + wrap1(x + q19x(i), nx);
        if (!solid[m]) touch = true;
    }
    cls[k] = touch ? CLS_BOUNDARY : CLS_INTERIOR;
}

__global__ void k3_cls2(uint8_t* cls, int nx, int ny, int nz, int pitch)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y, z = blockIdx.z;
    if (x >= nx || y >= ny) return;
    const size_t k = ((size_t)z * ny + y) * pitch + x;
    if (cls[k] != CLS_INTERIOR) return;
    for (int i = 1; i < 19; ++i) {
        int zz = z + q19z(i);
        if (zz < 0 || zz >= nz) continue;
        size_t m = ((size_t)zz * ny + wrap1(y + q19y(i), ny)) * pitch + wrap1(x + q19x(i), nx);
        if ((cls[m] & CLS_MASK) <= CLS_BOUNDARY) { cls[k] = CLS_GHOST; return; }
    }
}

__global__ void k3_cls3(uint8_t* cls, double* av, int nx, int ny, int nz, int pitch)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y, z = blockIdx.z;
    if (x >= nx || y >= ny) return;
    const size_t k = ((size_t)z * ny + y) * pitch + x;
    const uint8_t c = cls[k] & CLS_MASK;
    double a = 0.0;
    uint8_t flags = 0;
    if (c <= CLS_BOUNDARY) {
        int n[3] = {0, 0, 0};
        for (int i = 1; i < 19; ++i) {
            size_t m = ((size_t)(z + q19z(i)) * ny + wrap1(y + q19y(i), ny)) * pitch + wrap1(x + q19x(i), nx);
            const uint8_t cn = cls[m] & CLS_MASK;
            const int w36 = i <= 6 ? 2 : 1, eps = cn == CLS_FLUID ? 1 : 0;
            n[0] += w36 * q19x(i) * eps;
            n[1] += w36 * q19y(i) * eps;
            n[2] += w36 * q19z(i) * eps;
            if (cn > CLS_BOUNDARY) flags |= F_LINK;
        }
        if (n[0] | n[1] | n[2]) {
            a = sqrt((double)(n[0] * n[0] + n[1] * n[1] + n[2] * n[2])) / 12.0;
            flags |= F_WET;
        }
    }
    av[k] = a;
    cls[k] = c | flags;
}

template <typename C>
__global__ void k3_wet(const double* av, C* wet, size_t n, double coef)
{
    size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (k < n) wet[k] = (C)(av[k] * coef);
}

// ---- initial state (FP64 arithmetic) ----
// Outside r = R + 10 W the tanh profile is exactly 0 in FP64, so only the
// droplet's bounding box (periodic in x and y) is evaluated; a replacing
// call clears the field first.
// F32: the profile in FP32 (solves whose arithmetic is FP32; the FP64 tanh is
// slow on this part), else in FP64.
template <bool F32>
__global__ void k3_droplet(const uint8_t* cls, double* phi, int nx, int ny, int pitch, int xlo, int xw, int ylo,
                           int yw, int zlo, double x0, double y0, double z0, double R, double W)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = zlo + blockIdx.z;
    if (i >= xw || j >= yw) return;
    int x = (xlo + i) % nx, y = (ylo + j) % ny;
    if (x < 0) x += nx;
    if (y < 0) y += ny;
    const size_t k = ((size_t)z * ny + y) * pitch + x;
    if (!zeta_of(cls[k])) return;
    // periodic distances (fmod, exact, only for a distance of a period or more)
    double dx = fabs(x - x0), dy = fabs(y - y0);
    if (dx >= nx) dx = fmod(dx, (double)nx);
    if (dx > 0.5 * nx) dx = nx - dx;
    if (dy >= ny) dy = fmod(dy, (double)ny);
    if (dy > 0.5 * ny) dy = ny - dy;
    const double dz = z - z0, r2 = dx * dx + dy * dy + dz * dz;
    // beyond |R| + 10 W the profile is 0 in FP64 (tanh(-20) rounds to -1):
    // the bounding box's corners are skipped like the nodes outside it
    const double reach = fabs(R) + 10.0 * W;
    if (r2 > reach * reach) return;
    const double v = F32 ? (double)(0.5f + 0.5f * tanhf(2.0f * ((float)R - sqrtf((float)r2)) / (float)W))
                         : 0.5 + 0.5 * tanh(2.0 * (R - sqrt(r2)) / W);
    if (v > phi[k]) phi[k] = v;
}

__global__ void k3_ghost_init(const uint8_t* cls, double* phi, int nx, int ny, int nz, int pitch)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y, z = blockIdx.z;
    if (x >= nx || y >= ny) return;
    const size_t k = ((size_t)z * ny + y) * pitch + x;
    const uint8_t c = cls[k] & CLS_MASK;
    if (c == CLS_INTERIOR) { phi[k] = 0.0; return; }
    if (c != CLS_GHOST) return;
    double num = 0.0, den = 0.0;
    for (int dz = -1; dz <= 1; ++dz) {
        if (z + dz < 0 || z + dz >= nz) continue;
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                size_t m = ((size_t)(z + dz) * ny + wrap1(y + dy, ny)) * pitch + wrap1(x + dx, nx);
                if (zeta_of(cls[m])) { num += phi[m]; den += 1.0; }
            }
    }
    phi[k] = num / den;
}

template <int PREC>
__global__ void k3_init_pop(Args3<PREC> a, const double* phi0, double* mu0, Params q)
{
    using T = Store<PREC>;
    using C = typename T::C;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y, z = blockIdx.z;
    if (x >= a.nx || y >= a.ny) return;
    const int k = (z * a.ny + y) * a.pitch + x;
    for (int i = 0; i < 19; ++i) a.f_in[i * a.plane + k] = T::template st<0>(C(0));
    for (int i = 1; i < 7; ++i) a.g_in[i * a.plane + k] = T::template st<1>(C(0));
    a.g0_in[k] = T::g0_from_double(0.0);
    a.sprev[k] = C(0);
    const uint8_t code = a.cls[k];
    if (!zeta_of(code)) return;
    // mu of the initial field (Eq. chemical_potencial2) in the precision of the
    // step's arithmetic (FP64 for FP64 solves, FP32 otherwise: FP64 arithmetic
    // is slow on this part); phi itself stays FP64, so g_0 + sum g_i = phi0
    const double phd = phi0[k];
    const C ph = (C)phd;
    C gp[3] = {C(0), C(0), C(0)}, lap = C(0);
    for (int i = 1; i < 19; ++i) {
        const C v = (C)phi0[nbr(a, x, y, z, q19x(i), q19y(i), q19z(i))];
        const C w3 = C(3) * q19w<C>(i);
        gp[0] += w3 * C(q19x(i)) * v;
        gp[1] += w3 * C(q19y(i)) * v;
        gp[2] += w3 * C(q19z(i)) * v;
        lap += C(2) * w3 * (v - ph);
    }
    const C wet = (code & F_WET) ? a.wet[k] : C(0);
    const C mu = C(4) * (C)q.beta * ph * (ph - C(1)) * (ph - C(0.5)) - (C)q.kappa * lap - wet * (ph - ph * ph);
    mu0[k] = (double)mu;
    const C rho = (C)q.rho_g + (C)(q.rho_l - q.rho_g) * ph, h = C(0.5) / rho;
    a.sprev[k] = (mu * gp[0] * gp[0] + mu * gp[1] * gp[1] + mu * gp[2] * gp[2]) * h;
    a.g0_in[k] = T::g0_from_double(phd - 0.75 * q.alpha * (double)mu);
}

// g_i (i != 0) of the first pull: g_i^eq(mu) at x + c_i, or at x itself when
// x + c_i is not a zeta = 1 node (doubly-unknown rule), like the 2D init.
template <int PREC>
__global__ void k3_init_g(Args3<PREC> a, const double* mu0, double alpha)
{
    using T = Store<PREC>;
    using C = typename T::C;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y, z = blockIdx.z;
    if (x >= a.nx || y >= a.ny) return;
    const int k = (z * a.ny + y) * a.pitch + x;
    if (!zeta_of(a.cls[k])) return;
    for (int i = 1; i < 7; ++i) {
        int m = nbr(a, x, y, z, q19x(i), q19y(i), q19z(i));
        if (!zeta_of(a.cls[m])) m = k;
        a.g_in[i * a.plane + k] = T::template st<1>((C)(0.125 * alpha * mu0[m]));
    }
}

// FP64 mass: sum of pulled g over zeta = 1 nodes, block partials, fixed order
template <int PREC>
__global__ void __launch_bounds__(256) k3_mass(Args3<PREC> a, double* partial)
{
    __shared__ double sh[8];
    double acc = 0.0;
    const long long N = (long long)a.nx * a.ny * a.nz;
    for (long long t = blockIdx.x * 256LL + threadIdx.x; t < N; t += (long long)gridDim.x * 256) {
        const int x = (int)(t % a.nx), y = (int)((t / a.nx) % a.ny), z = (int)(t / ((long long)a.nx * a.ny));
        const int k = (z * a.ny + y) * a.pitch + x;
        const uint8_t c = a.cls[k];
        if (!zeta_of(c)) continue;
        const bool check = (c & F_LINK) != 0;
        double v = Store<PREC>::g0_double(a.g0_in[k]);
        v += (double)pull3<1, PREC>(a, a.g_in, x, y, z, k, check) + (double)pull3<2, PREC>(a, a.g_in, x, y, z, k, check);
        v += (double)pull3<3, PREC>(a, a.g_in, x, y, z, k, check) + (double)pull3<4, PREC>(a, a.g_in, x, y, z, k, check);
        v += (double)pull3<5, PREC>(a, a.g_in, x, y, z, k, check) + (double)pull3<6, PREC>(a, a.g_in, x, y, z, k, check);
        acc += v;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double r = threadIdx.x < 8 ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
        if (threadIdx.x == 0) partial[blockIdx.x] = r;
    }
}

__global__ void k3_sum(const double* partial, int n, double* out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += partial[i];
        *out = s;
    }
}


}  // namespace pfk3
using namespace pfk3;

namespace {

template <int PREC>
Args3<PREC> make3(pflbm3d_t* h, int in)
{
    using T = Store<PREC>;
    using C = typename T::C;
    Args3<PREC> a{};
    const size_t plane = (size_t)h->nz * h->ny * h->pitch;
    auto planes = [&](void* base, typename T::S*& f, typename T::S*& g, typename T::G0T*& g0) {
        f = (typename T::S*)base;
        g = f + 19 * plane;
        g0 = (typename T::G0T*)g;
    };
    planes(h->pop[in], a.f_in, a.g_in, a.g0_in);
    planes(h->pop[in ^ 1], a.f_out, a.g_out, a.g0_out);
    a.cls = h->cls;
    a.wet = (const C*)h->wet;
    a.sprev = (C*)h->sprev;
    a.phi = (C*)h->phi;
    a.nx = h->nx;
    a.ny = h->ny;
    a.nz = h->nz;
    a.pitch = h->pitch;
    a.plane = (int)plane;
    const Params& q = h->prm;
    a.beta4 = (C)(4.0 * q.beta);
    a.kappa = (C)q.kappa;
    a.rho_g = (C)q.rho_g;
    a.drho = (C)(q.rho_l - q.rho_g);
    a.omega_f = (C)(1.0 / q.tau_f);
    a.omega_g = (C)(1.0 / q.tau_g);
    a.force_pre = (C)(1.0 - 0.5 / q.tau_f);
    a.alpha = (C)q.alpha;
    a.dgdt = q.dgdt_mode;
    a.status = h->dstatus;
    {
        // the prefetch distance of k3_phi split into tiles along x, y and z of
        // its grid (grid3: 32 x 8 tiles, one z per CTA)
        const long long gx = (h->nx + 31) / 32, gy = (h->ny + 7) / 8, ahead = PFLBM3D_PHI_AHEAD;
        a.pf_dx = (int)(ahead % gx);
        a.pf_dy = (int)((ahead / gx) % gy);
        a.pf_dz = (int)(ahead / (gx * gy));
    }
    return a;
}

dim3 grid3(const pflbm3d_t* h) { return dim3((h->nx + 31) / 32, (h->ny + 7) / 8, h->nz); }

template <int PREC>
cudaError_t step3_prec(pflbm3d_t* h)
{
    Args3<PREC> a = make3<PREC>(h, h->cur);
    dim3 b(32, 8), g = grid3(h);
    if (h->fused) {
        const int chunks = (h->nz - 2 + h->fused_zc - 1) / h->fused_zc;
        dim3 gf((h->nx + TX - 1) / TX, (h->ny + TY - 1) / TY, chunks);
        k3_fused<PREC><<<gf, b, fused_smem_bytes<PREC>(), h->stream>>>(a, h->fused_zc, h->gflag);
        return cudaGetLastError();
    }
    k3_phi<PREC><<<g, b, 0, h->stream>>>(a);
    if (h->n_ghosts) k3_ghost<PREC><<<(h->n_ghosts + 255) / 256, 256, 0, h->stream>>>(a, h->ghosts, h->n_ghosts);
    k3_step<PREC, true><<<g, b, 0, h->stream>>>(a);
    return cudaGetLastError();
}

template <int PREC>
cudaError_t macro3_prec(pflbm3d_t* h, double* phi, double* u, double* p, float* fphi = nullptr, float* fu = nullptr,
                        float* fp = nullptr)
{
    Args3<PREC> a = make3<PREC>(h, h->cur);
    a.o_phi = phi;
    a.o_u = u;
    a.o_p = p;
    a.f_phi = fphi;
    a.f_u = fu;
    a.f_p = fp;
    dim3 b(32, 8), g = grid3(h);
    k3_phi<PREC><<<g, b, 0, h->stream>>>(a);
    if (h->n_ghosts) k3_ghost<PREC><<<(h->n_ghosts + 255) / 256, 256, 0, h->stream>>>(a, h->ghosts, h->n_ghosts);
    k3_step<PREC, false><<<g, b, 0, h->stream>>>(a);
    return cudaGetLastError();
}

template <int PREC>
cudaError_t init3_prec(pflbm3d_t* h)
{
    Args3<PREC> a = make3<PREC>(h, h->cur);
    dim3 b(32, 8), g = grid3(h);
    k3_ghost_init<<<g, b, 0, h->stream>>>(h->cls, h->phi0, h->nx, h->ny, h->nz, h->pitch);
    k3_init_pop<PREC><<<g, b, 0, h->stream>>>(a, h->phi0, h->mu0, h->prm);
    k3_init_g<PREC><<<g, b, 0, h->stream>>>(a, h->mu0, h->prm.alpha);
    return cudaGetLastError();
}

template <int PREC>
cudaError_t mass3_prec(pflbm3d_t* h, double* d_out)
{
    Args3<PREC> a = make3<PREC>(h, h->cur);
    k3_mass<PREC><<<kMassBlocks, 256, 0, h->stream>>>(a, h->red);
    k3_sum<<<1, 32, 0, h->stream>>>(h->red, kMassBlocks, d_out);
    return cudaGetLastError();
}


}  // namespace

namespace pfk3 {

cudaError_t launch_step(pflbm3d_t* h)
{
    return h->precision == PFLBM_FP64 ? step3_prec<PFLBM_FP64>(h) : step3_prec<PFLBM_FP32>(h);
}

cudaError_t launch_macro(pflbm3d_t* h, double* phi, double* u, double* p)
{
    return h->precision == PFLBM_FP64 ? macro3_prec<PFLBM_FP64>(h, phi, u, p) : macro3_prec<PFLBM_FP32>(h, phi, u, p);
}

cudaError_t launch_macro_f32(pflbm3d_t* h, float* phi, float* u, float* p)
{
    return h->precision == PFLBM_FP64 ? macro3_prec<PFLBM_FP64>(h, nullptr, nullptr, nullptr, phi, u, p)
                                      : macro3_prec<PFLBM_FP32>(h, nullptr, nullptr, nullptr, phi, u, p);
}

cudaError_t launch_init(pflbm3d_t* h)
{
    return h->precision == PFLBM_FP64 ? init3_prec<PFLBM_FP64>(h) : init3_prec<PFLBM_FP32>(h);
}

cudaError_t launch_mass(pflbm3d_t* h, double* d_out)
{
    return h->precision == PFLBM_FP64 ? mass3_prec<PFLBM_FP64>(h, d_out) : mass3_prec<PFLBM_FP32>(h, d_out);
}

cudaError_t launch_geometry(pflbm3d_t* h, double wet_coef)
{
    dim3 b(32, 8), g = grid3(h);
    k3_cls1<<<g, b, 0, h->stream>>>(h->solid, h->cls, h->nx, h->ny, h->nz, h->pitch);
    k3_cls2<<<g, b, 0, h->stream>>>(h->cls, h->nx, h->ny, h->nz, h->pitch);
    k3_cls3<<<g, b, 0, h->stream>>>(h->cls, h->av, h->nx, h->ny, h->nz, h->pitch);
    const size_t plane = (size_t)h->nz * h->ny * h->pitch;
    const unsigned nb = (unsigned)((plane + 255) / 256);
    if (h->precision == PFLBM_FP64)
        k3_wet<double><<<nb, 256, 0, h->stream>>>(h->av, (double*)h->wet, plane, wet_coef);
    else
        k3_wet<float><<<nb, 256, 0, h->stream>>>(h->av, (float*)h->wet, plane, wet_coef);
    return cudaGetLastError();
}

cudaError_t launch_ghost_collect(pflbm3d_t* h, int* count, int* list)
{
    dim3 b(32, 8), g = grid3(h);
    k3_ghost_collect<<<g, b, 0, h->stream>>>(h->cls, h->nx, h->ny, h->nz, h->pitch, count, list);
    return cudaGetLastError();
}

cudaError_t launch_ghost_flags(pflbm3d_t* h)
{
    const int tiles_x = (h->nx + TX - 1) / TX;
    const long long tiles = (long long)tiles_x * ((h->ny + TY - 1) / TY);
    k3_ghost_flags<<<dim3((unsigned)tiles, h->nz), 128, 0, h->stream>>>(h->cls, h->nx, h->ny, h->nz, h->pitch,
                                                                         tiles_x, h->gflag);
    return cudaGetLastError();
}

cudaError_t launch_droplet(pflbm3d_t* h, int xlo, int xw, int ylo, int yw, int zlo, int zn, double x0, double y0,
                           double z0, double R)
{
    dim3 b(32, 8), g((xw + 31) / 32, (yw + 7) / 8, zn);
    if (h->precision == PFLBM_FP64)
        k3_droplet<false><<<g, b, 0, h->stream>>>(h->cls, h->phi0, h->nx, h->ny, h->pitch, xlo, xw, ylo, yw, zlo, x0,
                                                  y0, z0, R, h->prm.W);
    else
        k3_droplet<true><<<g, b, 0, h->stream>>>(h->cls, h->phi0, h->nx, h->ny, h->pitch, xlo, xw, ylo, yw, zlo, x0,
                                                 y0, z0, R, h->prm.W);
    return cudaGetLastError();
}

cudaError_t fused_setup(int precision, size_t* smem_bytes, int* ctas_per_sm)
{
    const size_t sb = precision == PFLBM_FP64 ? fused_smem_bytes<PFLBM_FP64>() : fused_smem_bytes<PFLBM_FP32>();
    cudaError_t e = precision == PFLBM_FP64
        ? cudaFuncSetAttribute(k3_fused<PFLBM_FP64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb)
        : cudaFuncSetAttribute(k3_fused<PFLBM_FP32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb);
    if (e != cudaSuccess) return e;
    *smem_bytes = sb;
    return precision == PFLBM_FP64
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, k3_fused<PFLBM_FP64>, 256, sb)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, k3_fused<PFLBM_FP32>, 256, sb);
}

}  // namespace pfk3
