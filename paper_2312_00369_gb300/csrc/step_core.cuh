// step_core.cuh -- the per-node arithmetic of the time step, shared by every
// step kernel (single lattice and batched; populations pulled from global
// memory or from a shared-memory ring filled by TMA). Each kernel supplies
// the pulled populations and the phi tile; everything from there on -- the
// stencils, the chemical potential with the wetting term, the moments, both
// collisions and the stores -- is this one code, so all kernels round alike.
#pragma once

#include "storage.cuh"

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

// Stencils of Eqs. gradient and Laplace at phi-tile position (py, px).
template <typename C, int PW>
__device__ __forceinline__ void stencils(const C (*s_phi)[PW], int py, int px, C& gx, C& gy, C& lap)
{
    C c = s_phi[py][px];
    C E = s_phi[py][px + 1], W = s_phi[py][px - 1], N = s_phi[py + 1][px], Sx = s_phi[py - 1][px];
    C NE = s_phi[py + 1][px + 1], NW = s_phi[py + 1][px - 1], SW = s_phi[py - 1][px - 1], SE = s_phi[py - 1][px + 1];
    gx = fmadd(E - W, C(1) / C(3), ((NE + SE) - (NW + SW)) * (C(1) / C(12)));
    gy = fmadd(N - Sx, C(1) / C(3), ((NE + NW) - (SE + SW)) * (C(1) / C(12)));
    lap = fmadd((E + W) + (N + Sx), C(2) / C(3), fmadd((NE + NW) + (SE + SW), C(1) / C(6), c * (C(-10) / C(3))));
}

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

template <int PREC, int I, int O>
__device__ __forceinline__ void collide_f_pair(const StepArgs<PREC>& a, typename Store<PREC>::C fI,
                                               typename Store<PREC>::C fO, const PairK<typename Store<PREC>::C>& K,
                                               typename Store<PREC>::C ux, typename Store<PREC>::C uy,
                                               typename Store<PREC>::C Fx, typename Store<PREC>::C Fy,
                                               typename Store<PREC>::C drx, typename Store<PREC>::C dry, int k)
{
    using T = Store<PREC>;
    using C = typename T::C;
    static_assert(cx(O) == -cx(I) && cy(O) == -cy(I), "opposite pair");
    const C w = wgt<C>(I);
    const C cu = cdot<cx(I), cy(I)>(ux, uy);
    const C cF = cdot<cx(I), cy(I)>(Fx, Fy);
    const C cdr = cdot<cx(I), cy(I)>(drx, dry);
    // 16-bit work units f~ = f scale / w: the factor w becomes scale, which
    // the caller has folded into K
    C S = fmadd(cu, fmadd(K.c45, cu, K.pre3 * cdr), K.base);
    C A = fmadd(K.c3, cu, K.pre3 * cF);
    if constexpr (!T::kNorm) {
        S = w * S;
        A = w * A;
    }
    PFLBM_ST(a.out.f, I * a.plane + k, 9LL * a.plane, T::template stp<I>(fmadd(K.omf, fI, S + A)));
    PFLBM_ST(a.out.f, O * a.plane + k, 9LL * a.plane, T::template stp<O>(fmadd(K.omf, fO, S - A)));
}

// g_i (i != 0) collision and store; returns the storage rounding residual
// (population computed minus population stored) for the 16-bit formats.
template <int PREC, int I>
__device__ __forceinline__ typename Store<PREC>::C collide_g_dir(const StepArgs<PREC>& a,
                                                                 typename Store<PREC>::C g_i,
                                                                 typename Store<PREC>::C omg,
                                                                 typename Store<PREC>::C gadd, int k)
{
    using T = Store<PREC>;
    using C = typename T::C;
    // g*_i = (1 - omega_g) g_i + w_i (omega_g alpha mu + h_i src): gadd is the
    // second term, the same for the four axes and for the four diagonals
    const C v = fmadd(omg, g_i, gadd);
    const typename T::S s = T::template stp<I>(v);
    PFLBM_ST(a.out.g, I * a.plane + k, 9LL * a.plane, s);
    if (T::kAbsorb) return v - T::template ldp<I>(s);   // in work units
    return C(0);
}

// The time step of one node after its g has been pulled and the phi tile
// (with ghost values) is complete: chemical potential, coupling fields,
// moments, both collisions and the stores. (py, px) is the node's position
// in the phi tile, (gx, gy) its lattice coordinates; pull_f(f) fills the
// node's pulled f (called where the moments need it) and sprev(k) the
// u.grad(phi) history of the previous step at index k (called only with the
// (1/2) dG/dt term). With COLLIDE = false the macroscopic fields are written instead.
// Shared by every step kernel, so the arithmetic (and its rounding) is the
// same in all of them. VV: 0 uniform tau_f, 1 variable viscosity, 2 decided
// by a.varvisc.
template <int PREC, bool COLLIDE, int VV, int PW, typename PullF, typename SprevF>
__device__ __forceinline__ void node_step(const StepArgs<PREC>& a, uint8_t code, const typename Store<PREC>::C (*s_phi)[PW],
                                          int py, int px, int gx, int gy, const typename Store<PREC>::C g[9],
                                          typename Store<PREC>::G0T g0raw, PullF&& pull_f, SprevF&& sprev)
{
    using T = Store<PREC>;
    using C = typename T::C;
    C f[9];
    const int k = gy * a.pitch + gx;
    if (!zeta_of(code)) {
        if (!COLLIDE) {
            const size_t o = (size_t)gy * a.nx + gx;
            const long long no = (long long)a.nx * a.ny;
            if (a.o_phi) PFLBM_ST(a.o_phi, o, no, (double)s_phi[py][px]);
            if (a.o_u) { PFLBM_ST(a.o_u, 2 * o, 2 * no, 0.0); PFLBM_ST(a.o_u, 2 * o + 1, 2 * no, 0.0); }
            if (a.o_p) PFLBM_ST(a.o_p, o, no, 0.0);
            if (a.f_phi) PFLBM_ST(a.f_phi, o, no, (float)s_phi[py][px]);
            if (a.f_u) { PFLBM_ST(a.f_u, 2 * o, 2 * no, 0.0f); PFLBM_ST(a.f_u, 2 * o + 1, 2 * no, 0.0f); }
            if (a.f_p) PFLBM_ST(a.f_p, o, no, 0.0f);
        }
        return;
    }

    // ---- chemical potential (Eq. chemical_potencial2) ----
    C gpx, gpy, lap;
    stencils<C, PW>(s_phi, py, px, gpx, gpy, lap);
    const C ph = s_phi[py][px];
    const C wet = (code & F_WET) ? PFLBM_LD(a.wet, k, a.plane) : C(0);
    const C mu = fmadd(-wet, fmadd(-ph, ph, ph), fmadd(-a.kappa, lap, a.beta4 * ph * (ph - C(1)) * (ph - C(0.5))));

    // ---- coupling fields (Sec. 2.1.1): F = F_s + F_b, F_s = mu grad(phi), F_b = rho g ----
    const C rho = fmadd(a.drho, ph, a.rho_g);
    const C drx = a.drho * gpx, dry = a.drho * gpy;
    const C Fx = fmadd(mu, gpx, rho * a.gx), Fy = fmadd(mu, gpy, rho * a.gy);

    // ---- hydrodynamic moments (Sec. 2.1.2) ----
    pull_f(f);
    C mx, my;
    if constexpr (T::kNorm) {
        mx = fmadd(T::template unit<1>(), f[1] - f[3], T::template unit<5>() * ((f[5] - f[6]) + (f[8] - f[7])));
        my = fmadd(T::template unit<1>(), f[2] - f[4], T::template unit<5>() * ((f[5] + f[6]) - (f[7] + f[8])));
    } else {
        mx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
        my = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
    }
    const C inv_rho = C(1) / rho;
    const C ux = fmadd(C(0.5), Fx, mx) * inv_rho;
    const C uy = fmadd(C(0.5), Fy, my) * inv_rho;
    const C uu = fmadd(ux, ux, uy * uy);
    const C fsum = sum_pop<PREC>(f);
    // p = c_s^2/(1 - w_0) [sum_{i!=0} f_i + u.grad(rho)/2 + rho s_0(u)], s_0 = -w_0 (3/2) u^2
    const C p = C(0.6) * fmadd(-(rho * (C(2) / C(3))), uu, fmadd(C(0.5), fmadd(ux, drx, uy * dry), fsum));

    if (!COLLIDE) {
        size_t o = (size_t)gy * a.nx + gx;
        const long long no = (long long)a.nx * a.ny;
        if (a.o_phi) PFLBM_ST(a.o_phi, o, no, (double)ph);
        if (a.o_u) { PFLBM_ST(a.o_u, 2 * o, 2 * no, (double)ux); PFLBM_ST(a.o_u, 2 * o + 1, 2 * no, (double)uy); }
        if (a.o_p) PFLBM_ST(a.o_p, o, no, (double)p);
        if (a.f_phi) PFLBM_ST(a.f_phi, o, no, (float)ph);
        if (a.f_u) { PFLBM_ST(a.f_u, 2 * o, 2 * no, (float)ux); PFLBM_ST(a.f_u, 2 * o + 1, 2 * no, (float)uy); }
        if (a.f_p) PFLBM_ST(a.f_p, o, no, (float)p);
        return;
    }
    if (!(uu < C(0.09))) atomicOr(a.status, 1);
    // relaxation of f: uniform, or tau_f(x) = nu(phi) / c_s^2 + 1/2 with
    // nu(phi) = phi (nu_l - nu_g) + nu_g (Secs. 2.1.1, 2.1.2)
    C omega_f = a.omega_f, force_pre = a.force_pre;
    if (VV == 1 || (VV == 2 && a.varvisc)) {
        omega_f = C(1) / fmadd(a.dtau3, ph, a.tau_g3h);
        force_pre = fmadd(C(-0.5), omega_f, C(1));
    }

    // ---- f collision: f* = f + (f^eq - f)/tau_f + F_i ----
    {
        C feq0 = fmadd(-(rho * (wgt<C>(0) * C(1.5))), uu, (C(-5) / C(3)) * p);
        if constexpr (T::kNorm) feq0 = feq0 * (C(1) / T::template unit<0>());
        PFLBM_ST(a.out.f, k, 9LL * a.plane, T::template stp<0>(fmadd(omega_f, feq0 - f[0], f[0])));
    }
    {
        PairK<C> K;
        K.base = omega_f * fmadd(-(C(1.5) * rho), uu, C(3) * p);
        K.c45 = omega_f * C(4.5) * rho;
        K.c3 = omega_f * C(3) * rho;
        K.pre3 = C(3) * force_pre;
        K.omf = C(1) - omega_f;
        if constexpr (T::kNorm) {          // scale is a power of two: exact
            K.base = K.base * T::scale();
            K.c45 = K.c45 * T::scale();
            K.c3 = K.c3 * T::scale();
            K.pre3 = K.pre3 * T::scale();
        }
        collide_f_pair<PREC, 1, 3>(a, f[1], f[3], K, ux, uy, Fx, Fy, drx, dry, k);
        collide_f_pair<PREC, 2, 4>(a, f[2], f[4], K, ux, uy, Fx, Fy, drx, dry, k);
        collide_f_pair<PREC, 5, 7>(a, f[5], f[7], K, ux, uy, Fx, Fy, drx, dry, k);
        collide_f_pair<PREC, 6, 8>(a, f[6], f[8], K, ux, uy, Fx, Fy, drx, dry, k);
    }

    // ---- g collision: g* = g + (g^eq - g)/tau_g + (3/2) G_i(t) - (1/2) G_i(t-1) ----
    const C s_now = fmadd(ux, gpx, uy * gpy);
    const C src = a.dgdt ? s_now : fmadd(C(1.5), s_now, C(-0.5) * sprev(k));
    const C am = a.alpha * mu;
    const C omg = C(1) - a.omega_g, oam = a.omega_g * am;
    // h = -1/2 on the axes, 1 on the diagonals; in the 16-bit work units the
    // factor w_i is scale for every direction
    const C g_ax = (T::kNorm ? T::scale() : wgt<C>(1)) * fmadd(C(-0.5), src, oam);
    const C g_dg = (T::kNorm ? T::scale() : wgt<C>(5)) * (oam + src);
    C r_ax = collide_g_dir<PREC, 1>(a, g[1], omg, g_ax, k);
    r_ax += collide_g_dir<PREC, 2>(a, g[2], omg, g_ax, k);
    r_ax += collide_g_dir<PREC, 3>(a, g[3], omg, g_ax, k);
    r_ax += collide_g_dir<PREC, 4>(a, g[4], omg, g_ax, k);
    C r_dg = collide_g_dir<PREC, 5>(a, g[5], omg, g_dg, k);
    r_dg += collide_g_dir<PREC, 6>(a, g[6], omg, g_dg, k);
    r_dg += collide_g_dir<PREC, 7>(a, g[7], omg, g_dg, k);
    r_dg += collide_g_dir<PREC, 8>(a, g[8], omg, g_dg, k);
    // storage rounding residual in population units (0 for FP32 / FP64)
    const C resid = T::kAbsorb ? fmadd(T::template unit<1>(), r_ax, T::template unit<5>() * r_dg) : C(0);
    {
        // g_0^eq - g_0 = sum_{i!=0} g_i - (1 - w_0) alpha mu (Eq. H_i); in the
        // 16-bit formats g_0 also takes back what rounding removed from g_1..g_8
        const C d0 = fmadd(a.omega_g, fmadd(-(C(1) - wgt<C>(0)), am, sum_pop<PREC>(g)), (wgt<C>(0) * C(-2)) * src);
        PFLBM_ST(a.out.g0, k, a.plane, T::g0_add(g0raw, T::kAbsorb ? d0 + resid : d0, a.status));
    }
    if (!a.dgdt) PFLBM_ST(a.sprev, k, a.plane, s_now);
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
