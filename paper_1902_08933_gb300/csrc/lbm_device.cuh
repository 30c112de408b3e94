// lbm_device.cuh -- device code of the phase-field lattice Boltzmann step
// (arXiv:1902.08933, Sec. 3), shared by the per-precision translation units.
//
// Data layout (structure of arrays, one plane per population direction):
//   pop[i * S + base + y * nx + x],  S = plane stride (all instances), base = the
//   instance's first cell. The state between steps is the set of post-streaming
//   populations h_i(x, t), g_i(x, t) (as in Eqs. 10 and 24, left-hand side), the
//   product phi*u of the previous step (for Eq. 14) and the pressure p of the
//   previous step (for grad p, reading Q2). g_0 is stored shifted by rho_0, i.e.
//   the kernel works with rho_0 = 0: rho_0 enters only g_0 and cancels from every
//   output (Eq. 33, App. B).
//
// Fused step kernel (one launch per time step): a thread block owns a strip of
// TX columns and marches over a run of rows. Per output row Y it
//   A. loads the populations h of the lead row Y + 2d (aligned loads) and forms
//      phi = sum_i h_i (Eq. 18) over the strip plus a 2-column halo, keeping
//      h in shared memory for the collision two rows later; loads p of row Y + d;
//   B. forms mu (Eq. 8, Laplacian of Eq. 30b) of row Y + d from the phi ring;
//   C. collides row Y: stencils of phi, mu, p (Eq. 30), forces, velocity
//      (Eq. 27a), pressure (Eq. 28/29), g^eq (Eq. 33), G_i (Eq. 34), h^eq
//      (Eq. 11), R_i (Eq. 14), BGK updates (Eqs. 24, 10), and pushes the new
//      populations to their neighbours (periodic or halfway bounce-back).
// Every population is read from HBM once per step (halo columns aside) and
// written once; phi and mu never leave shared memory.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "lbm_internal.h"

namespace lbm {

// ---------------------------------------------------------------------------
// D2Q9 lattice (Sec. 2.2): order (0,0),(1,0),(0,1),(-1,0),(0,-1),(1,1),(-1,1),
// (-1,-1),(1,-1); weights 4/9, 1/9 (axes), 1/36 (diagonals); c_s^2 = 1/3.
__host__ __device__ constexpr int cx_of(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int cy_of(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__host__ __device__ constexpr int opp_of(int i) {
    return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 5 + 2) % 4) + 5);
}
template <typename R>
__host__ __device__ constexpr R w_of(int i) {
    return i == 0 ? R(4) / R(9) : (i <= 4 ? R(1) / R(9) : R(1) / R(36));
}

// ---------------------------------------------------------------------------
// Storage forms (enum order of include/lbm.h):
//   0 LBM_F64      everything FP64.
//   1 LBM_F32      everything FP32.
//   2 LBM_F32_G16  h_1..8 FP32, g FP16 (scaled), aux FP32, h_0 conservative.
//   3 LBM_F32_H16  h_1..8 FP16 (scaled), g FP16 (scaled), aux FP32, h_0 conservative.
//   4 LBM_F32_C    h_1..8 FP32, g FP32, aux FP32, h_0 conservative.
//   5 LBM_F32_CC   form 4, and mu formed from the two-float phi ("comp").
// "comp" (form 5): the paired kernels also form mu from phi = hi + lo
// (compensated stencil, chem_pot2). The FP16-storage forms do not offer it:
// their storage rounding dominates, and the extra stencil cost them 5-6 %.
// "Conservative h_0": h_0 is kept as an unevaluated sum of two floats (hi + lo)
// in a plane of its own and, after each collision, set to phi minus the stored
// (rounded) h_1..h_8, with error-free FP32 transformations. The stored
// populations of a cell then sum to phi to about 2^-48, so the storage rounding
// cannot create or destroy phi: the global sum of phi is conserved although the
// arithmetic is FP32 (plain FP32 drifts by ~2^-24 per step where phi ~ 1 sits in
// h_0 and rounds the same way every step).
template <int FORM> struct Form;
template <> struct Form<0> {
    using R = double; using HT = double; using GT = double; using AT = double;
    static constexpr bool h16 = false, g16 = false, cons = false, comp = false;
};
template <> struct Form<1> {
    using R = float; using HT = float; using GT = float; using AT = float;
    static constexpr bool h16 = false, g16 = false, cons = false, comp = false;
};
template <> struct Form<2> {
    using R = float; using HT = float; using GT = __half; using AT = float;
    static constexpr bool h16 = false, g16 = true, cons = true, comp = false;
};
template <> struct Form<3> {
    using R = float; using HT = __half; using GT = __half; using AT = float;
    static constexpr bool h16 = true, g16 = true, cons = true, comp = false;
};
template <> struct Form<4> {
    using R = float; using HT = float; using GT = float; using AT = float;
    static constexpr bool h16 = false, g16 = false, cons = true, comp = false;
};
template <> struct Form<5> {
    using R = float; using HT = float; using GT = float; using AT = float;
    static constexpr bool h16 = false, g16 = false, cons = true, comp = true;
};

template <typename T, typename R> __device__ __forceinline__ R ldr(const T* p);
template <> __device__ __forceinline__ double ldr<double, double>(const double* p) { return *p; }
template <> __device__ __forceinline__ float ldr<float, float>(const float* p) { return *p; }
template <> __device__ __forceinline__ float ldr<__half, float>(const __half* p) {
    return __half2float(*p);
}
template <typename T, typename R> __device__ __forceinline__ void str(T* p, R v);
template <> __device__ __forceinline__ void str<double, double>(double* p, double v) { *p = v; }
template <> __device__ __forceinline__ void str<float, float>(float* p, float v) { *p = v; }
template <> __device__ __forceinline__ void str<__half, float>(__half* p, float v) {
    *p = __float2half_rn(v);
}

// Error-free transformations (Knuth's TwoSum, Dekker's Fast2Sum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {  // |a| >= |b|
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

// Population access through the storage form. For conservative forms plane 0 of
// h is a float2 plane (hi, lo) of its own and planes 1..8 sit at (i - 1) * S.
template <class F>
struct PopIO {
    using R = typename F::R;
    using HT = typename F::HT;
    using GT = typename F::GT;
    const HT* hin; HT* hout; const float2* h0in; float2* h0out;
    const GT* gin; GT* gout;
    long long S;
    R hs, ihs, gs, igs;    // storage scales and their inverses

    __device__ __forceinline__ long long hoff(int i) const {
        return (long long)(F::cons ? i - 1 : i) * S;
    }
    // h_i for i >= 1 (and i = 0 for non-conservative forms)
    __device__ __forceinline__ R load_h(int i, long long c) const {
        if constexpr (F::h16) return ldr<HT, R>(hin + hoff(i) + c) * ihs;
        else return ldr<HT, R>(hin + hoff(i) + c);
    }
    __device__ __forceinline__ float2 load_h0(long long c) const { return h0in[c]; }
    // the value of h_i (i >= 1) as it will be read back after storage
    __device__ __forceinline__ R round_h(R v) const {
        if constexpr (F::h16) return __half2float(__float2half_rn(v * hs)) * ihs;
        else return v;
    }
    __device__ __forceinline__ void store_h(int i, long long c, R v) const {
        if constexpr (F::h16) str<HT, R>(hout + hoff(i) + c, v * hs);
        else str<HT, R>(hout + hoff(i) + c, v);
    }
    __device__ __forceinline__ void store_h0(long long c, float2 v) const { h0out[c] = v; }
    __device__ __forceinline__ R load_g(int i, long long c) const {
        if constexpr (F::g16) return ldr<GT, R>(gin + (long long)i * S + c) * igs;
        else return ldr<GT, R>(gin + (long long)i * S + c);
    }
    __device__ __forceinline__ void store_g(int i, long long c, R v) const {
        if constexpr (F::g16) str<GT, R>(gout + (long long)i * S + c, v * gs);
        else str<GT, R>(gout + (long long)i * S + c, v);
    }
    // phi = sum_i h_i (Eq. 18) of cell c; for conservative forms also the low
    // part of phi (phi ~ hi + lo). Summation order: h_0 + h_1 + ... + h_8.
    __device__ __forceinline__ R phi_of(long long c, R hv[9], R& phi_lo) const {
        if constexpr (F::cons) {
            R s8 = R(0);
#pragma unroll
            for (int i = 1; i < 9; ++i) { hv[i] = load_h(i, c); s8 += hv[i]; }
            const float2 h0 = load_h0(c);
            float s, e, hi, lo;
            two_sum(h0.x, s8, s, e);
            fast_two_sum(s, e + h0.y, hi, lo);
            hv[0] = hi - s8;        // h_0 as seen by the arithmetic (not stored)
            phi_lo = lo;
            return hi;
        } else {
#pragma unroll
            for (int i = 0; i < 9; ++i) hv[i] = load_h(i, c);
            R phi = hv[0];
#pragma unroll
            for (int i = 1; i < 9; ++i) phi += hv[i];
            phi_lo = R(0);
            return phi;
        }
    }
    // h_0 after the collision for conservative forms: (phi_hi + phi_lo) - sum of the
    // stored h_1..8, as a normalised float pair.
    __device__ __forceinline__ float2 conservative_h0(float phi_hi, float phi_lo, float rest) const {
        float s, e, hi, lo;
        two_sum(phi_hi, -rest, s, e);
        fast_two_sum(s, e + phi_lo, hi, lo);
        return make_float2(hi, lo);
    }
};

// ---------------------------------------------------------------------------
// Per-instance constants in the arithmetic type.
// Reciprocal: FP32 uses the hardware approximation (max 2 ulp, __fdividef); FP64
// keeps the IEEE division so that the FP64 form tracks the oracle to round-off.
__device__ __forceinline__ float rcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }

template <typename R>
struct Consts {
    int nx, ny, walls, qim, pscheme, sforce, visc, uniform_nu;
    long long base;
    R tgm0, inv_tau_g0;   // tau_g - 1/2 and 1/tau_g when nu_A = nu_B (inverse-linear model)
    R rho_A, rho_B, drho, inv_nu_A, inv_nu_B, mu_A, mu_B, beta, kappa, eta, gammaM;
    R inv_tau_h, src_h;   // 1/tau_h and 1 - 1/(2 tau_h)
    R force_x, force_y, gravity;
    R hs, ihs, gs, igs;

    __device__ __forceinline__ void load(const DevInst& P) {
        nx = P.nx; ny = P.ny; walls = P.walls; qim = P.qim; pscheme = P.pscheme;
        sforce = P.sforce; visc = P.visc; base = P.base; uniform_nu = P.uniform_nu;
        tgm0 = R(P.tgm0); inv_tau_g0 = R(P.inv_tau_g0);
        rho_A = R(P.rho_A); rho_B = R(P.rho_B); drho = R(P.drho);
        inv_nu_A = R(P.inv_nu_A); inv_nu_B = R(P.inv_nu_B); mu_A = R(P.mu_A); mu_B = R(P.mu_B);
        beta = R(P.beta); kappa = R(P.kappa); eta = R(P.eta); gammaM = R(P.gammaM);
        inv_tau_h = R(P.inv_tau_h); src_h = R(1) - R(0.5) * R(P.inv_tau_h);
        force_x = R(P.force_x); force_y = R(P.force_y); gravity = R(P.gravity);
        hs = R(P.h_scale); ihs = R(1.0 / P.h_scale); gs = R(P.g_scale); igs = R(1.0 / P.g_scale);
    }
};

// ---------------------------------------------------------------------------
// Value types of the cell arithmetic: double, float, or F2 -- two cells' FP32
// values in the two lanes of a float2, computed with the packed FP32 instructions
// of sm_100+ (FFMA2 / FADD2 / FMUL2), so one instruction serves two cells. The
// cell functions below are written once for all three; constants come in the
// scalar type S of the instance constants.
struct F2 {
    float2 v;
    F2() = default;
    __device__ __forceinline__ F2(float s) : v(make_float2(s, s)) {}
    __device__ __forceinline__ F2(float a, float b) : v(make_float2(a, b)) {}
    __device__ __forceinline__ explicit F2(float2 w) : v(w) {}
};
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return F2(__fadd2_rn(a.v, b.v)); }
// a - b as a + (-1) b: the product is exact, so this rounds once, like a subtraction
__device__ __forceinline__ F2 operator-(F2 a, F2 b) {
    return F2(__ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v));
}
__device__ __forceinline__ F2 operator-(F2 a) { return F2(__fmul2_rn(a.v, make_float2(-1.f, -1.f))); }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return F2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator*(float s, F2 b) { return F2(s) * b; }
__device__ __forceinline__ F2 operator*(F2 a, float s) { return a * F2(s); }
__device__ __forceinline__ F2 operator+(F2 a, float s) { return a + F2(s); }
__device__ __forceinline__ F2 operator+(float s, F2 b) { return F2(s) + b; }
__device__ __forceinline__ F2 operator-(F2 a, float s) { return a - F2(s); }
__device__ __forceinline__ F2 operator-(float s, F2 b) { return F2(s) - b; }

template <typename V> struct ScalarOf { using type = V; };
template <> struct ScalarOf<F2> { using type = float; };

// a * b + c (one FFMA2 for F2; the compiler contracts the scalar form)
template <typename V>
__device__ __forceinline__ V fmadd(V a, V b, V c) { return a * b + c; }
__device__ __forceinline__ F2 fmadd(F2 a, F2 b, F2 c) { return F2(__ffma2_rn(a.v, b.v, c.v)); }
__device__ __forceinline__ F2 rcp(F2 x) { return F2(rcp(x.v.x), rcp(x.v.y)); }
// step dynamic viscosity of Sec. 4.3: a where phi >= 1/2, else b
template <typename V, typename S>
__device__ __forceinline__ V step_pick(V phi, S a, S b) { return phi >= V(0.5) ? V(a) : V(b); }
__device__ __forceinline__ F2 step_pick(F2 phi, float a, float b) {
    return F2(phi.v.x >= 0.5f ? a : b, phi.v.y >= 0.5f ? a : b);
}
// c . (x, y) for a lattice direction c = (cx, cy) with components in {-1, 0, 1};
// cx, cy are compile-time after unrolling, so this folds to one add or a copy.
template <typename V>
__device__ __forceinline__ V cdot(int cx, int cy, V x, V y) {
    if (cx == 0) return cy > 0 ? y : -y;
    if (cy == 0) return cx > 0 ? x : -x;
    if (cx > 0) return cy > 0 ? x + y : x - y;
    return cy > 0 ? y - x : -(x + y);
}

// Chemical potential, Eq. 8.
template <typename V, typename S>
__device__ __forceinline__ V chem_pot(const Consts<S>& C, V phi, V lap_phi) {
    return V(S(4) * C.beta) * phi * (phi - V(S(1))) * (phi - V(S(0.5))) - V(C.kappa) * lap_phi;
}

// Chemical potential, Eq. 8, for phi given as an unevaluated sum hi + lo (the
// conservative forms carry phi to about 2^-48): phi - 1 and phi - 1/2 are formed
// from hi first, exact where they cancel (Sterbenz), then corrected by lo, so the
// double-well term keeps FP32 relative precision in the bulk phases where it is
// small; lap_phi is the Laplacian of hi plus that of lo.
template <typename V, typename S>
__device__ __forceinline__ V chem_pot2(const Consts<S>& C, V hi, V lo, V lap_phi) {
    const V pm1 = (hi - V(S(1))) + lo, pmh = (hi - V(S(0.5))) + lo;
    return V(S(4) * C.beta) * (hi + lo) * pm1 * pmh - V(C.kappa) * lap_phi;
}

// 3x3 neighbourhood z[dy+1][dx+1] of a field around a cell.
template <typename V>
struct Nbr {
    using S = typename ScalarOf<V>::type;
    V z[3][3];
    // Isotropic gradient, Eq. 30a: sum_{i!=0} w_i c_i z(x + c_i) / c_s^2.
    __device__ __forceinline__ void grad(V& gx, V& gy) const {
        const V w1 = V(S(3) / S(9)), w2 = V(S(3) / S(36));   // w_i / c_s^2
        gx = fmadd(w1, z[1][2] - z[1][0], w2 * ((z[2][2] - z[2][0]) + (z[0][2] - z[0][0])));
        gy = fmadd(w1, z[2][1] - z[0][1], w2 * ((z[2][2] - z[0][2]) + (z[2][0] - z[0][0])));
    }
    // Isotropic Laplacian, Eq. 30b: sum_{i!=0} 2 w_i (z(x + c_i) - z(x)) / c_s^2.
    __device__ __forceinline__ V lap() const {
        const V c = z[1][1];
        const V a = (z[1][2] - c) + (z[2][1] - c) + (z[1][0] - c) + (z[0][1] - c);
        const V d = (z[2][2] - c) + (z[2][0] - c) + (z[0][0] - c) + (z[0][2] - c);
        return fmadd(V(S(6) / S(9)), a, V(S(6) / S(36)) * d);
    }
};

// Macroscopic stage of one cell (steps 1-6 of the time step): inputs are the
// post-streaming g, phi, mu and the stencils of phi, mu and p_prev.
template <typename V>
struct Macro {
    V rho, ux, uy, Fx, Fy, Ftx, Fty, S, S1, tgm /* tau_g - 1/2 */, inv_tau_g, p;
};

// GSC: the g values come in multiplied by the FP16 storage scale gs of the
// instance (as they are stored). gs is a power of two, and multiplying by a power
// of two commutes exactly with every rounded operation (no value here comes near
// the FP32 overflow or subnormal range), so un-scaling the three sums that use g
// (j_x, j_y, the sum of Eq. 28) gives bit for bit what un-scaling every g_i would.
template <bool GSC = false, typename V, typename S>
__device__ __forceinline__ Macro<V> macroscopic(const Consts<S>& C, const V g[9], V phi, V mu,
                                                V gphix, V gphiy, V gmux, V gmuy, V lapmu,
                                                V gpx, V gpy) {
    Macro<V> m;
    m.rho = fmadd(phi, V(C.drho), V(C.rho_B));         // Eq. 3aa (phi_B = 0)
    const V drx = V(C.drho) * gphix, dry = V(C.drho) * gphiy;   // grad rho
    m.S1 = C.qim ? V(-C.gammaM) * lapmu : V(S(0));     // Sec. 3.2.1
    V Fsx, Fsy;                                        // surface tension
    if (C.sforce == 0) { Fsx = mu * gphix; Fsy = mu * gphiy; }
    else { Fsx = -(phi * gmux); Fsy = -(phi * gmuy); }
    m.Fx = Fsx + V(C.force_x);
    m.Fy = fmadd(m.rho - V(C.rho_A), V(-C.gravity), Fsy + V(C.force_y));   // buoyancy, Sec. 4.4
    V jx = (g[1] - g[3]) + (g[5] - g[6]) + (g[8] - g[7]);
    V jy = (g[2] - g[4]) + (g[5] + g[6]) - (g[7] + g[8]);
    if constexpr (GSC) {
        jx = jx * V(C.igs);
        jy = jy * V(C.igs);
    }
    const V inv_rho = rcp(m.rho);
    m.ux = fmadd(V(S(0.5)), m.Fx, jx) * inv_rho;      // Eq. 27a
    m.uy = fmadd(V(S(0.5)), m.Fy, jy) * inv_rho;
    m.S = fmadd(m.ux, drx, fmadd(m.uy, dry, m.rho * m.S1));   // S = u.grad(rho) + rho S1
    if (C.uniform_nu) {                                // nu_A = nu_B: constant tau_g
        m.tgm = V(C.tgm0);
        m.inv_tau_g = V(C.inv_tau_g0);
    } else {                                           // viscosity, Sec. 3.2.2 / 4.3
        V nu;
        if (C.visc == 0) nu = rcp(fmadd(phi, V(C.inv_nu_A - C.inv_nu_B), V(C.inv_nu_B)));
        else nu = step_pick(phi, C.mu_A, C.mu_B) * inv_rho;
        m.tgm = V(S(3)) * nu;                          // tau_g - 1/2 = nu / c_s^2
        m.inv_tau_g = rcp(m.tgm + V(S(0.5)));
    }
    m.Ftx = fmadd(drx, V(S(1) / S(3)), m.Fx - gpx);   // F~ = F - grad(p - rho c_s^2)
    m.Fty = fmadd(dry, V(S(1) / S(3)), m.Fy - gpy);
    const S w0 = w_of<S>(0);
    V G0 = V(S(0));
    if (C.pscheme == 0) {         // simplified G_0 printed after Eq. 34
        const V uFp = fmadd(m.ux, m.Fx - gpx, m.uy * (m.Fy - gpy));
        G0 = V(w0) * fmadd(V(S(0.5)) * m.rho, m.S1, V(S(-3)) * uFp);
    } else if (C.pscheme == 1) {  // Eq. 34 at i = 0
        const V uFt = fmadd(m.ux, m.Ftx, m.uy * m.Fty);
        G0 = V(w0) * (fmadd(V(S(-3)), uFt, m.S) - m.rho * m.S1);
    }
    V sum_g = (((g[1] + g[2]) + (g[3] + g[4])) + ((g[5] + g[6]) + (g[7] + g[8])));
    if constexpr (GSC) sum_g = sum_g * V(C.igs);
    const V uu = fmadd(m.ux, m.ux, m.uy * m.uy);
    // Eq. 28 (Eq. 29 for the previous scheme): c_s^2 / (1 - w0) = 3/5, s_0 = -1.5 w0 u.u
    m.p = V(S(0.6)) * fmadd(m.tgm, G0, fmadd(m.rho * V(S(-1.5) * w0), uu, fmadd(V(S(0.5)), m.S, sum_g)));
    return m;
}

// ---------------------------------------------------------------------------
// Collision of one cell: g by Eq. 24 with g^eq of Eq. 33 (rho_0 = 0) and G_i of
// Eq. 34; h by Eq. 10 with h^eq of Eq. 11 and R_i of Eq. 14. Opposite directions
// i and j (c_j = -c_i) share the even parts of s_i, G_i and h^eq and differ in
// the sign of the odd parts, so each pair is formed once:
//   s_i   = w (3 c.u + 4.5 (c.u)^2 - 1.5 u.u)
//   G_i   = w [S + 3 c.F + 4.5 (2 (c.u)(c.F~) - (2/3) u.F~) + 1.5 (|c|^2 - 2/3) rho S1]
//   h^eq_i = w (eta mu + 3 c.(phi u)),  R_i = (1 - 1/(2 tau_h)) 3 w c.d_t(phi u).
// The collision written once, handing each result to emit(i, g*_i, h*_i) as soon
// as its pair of directions is formed (rest direction first), so callers that
// store right away keep few values alive.
// GSC / HSC: g / h come in and go out in the units they are stored in, i.e.
// multiplied by the FP16 storage scale gs / hs (powers of two). The scale is
// folded into per-cell factors (the relaxation weights of g; eta mu, phi u and
// the R_i constant of h), which gives bit for bit the scaled result of the
// unscaled arithmetic (see macroscopic) at a few multiplies a cell instead of
// two per stored value.
template <bool GSC = false, bool HSC = false, typename V, typename S, typename Emit>
__device__ __forceinline__ void collide_emit(const Consts<S>& C, const Macro<V>& m, V phi, V mu,
                                             V ddx, V ddy, const V g[9], const V h[9], Emit&& emit) {
    auto hsc = [&](S k) {   // a constant of the h update in the units h is stored in
        if constexpr (HSC) return k * C.hs;
        else return k;
    };
    const V uu = fmadd(m.ux, m.ux, m.uy * m.uy);
    const V uFt = fmadd(m.ux, m.Ftx, m.uy * m.Fty);
    const V om = m.inv_tau_g, om1 = V(S(1)) - om;
    const V gsrc = fmadd(V(S(-0.5)), om, V(S(1)));
    V omg = om, gsrcg = gsrc;   // weights of g^eq and G_i in the units g is stored in
    if constexpr (GSC) {
        omg = om * V(C.gs);
        gsrcg = gsrc * V(C.gs);
    }
    const V omh = V(C.inv_tau_h), omh1 = V(S(1) - C.inv_tau_h);
    const V p3 = V(S(3)) * m.p;
    const V rS1 = m.rho * m.S1;
    const V etamu = V(hsc(C.eta)) * mu;
    V phih = phi;
    if constexpr (HSC) phih = phi * V(C.hs);
    const V phiux = phih * m.ux, phiuy = phih * m.uy;
    const V uu15 = V(S(-1.5)) * uu;
    // rest direction (c = 0): G_0 = w0 (S - 3 u.F~ - rho S1), R_0 = 0
    {
        const S w0 = w_of<S>(0);
        const V geq = fmadd(V(w0 - S(1)), p3, m.rho * (V(w0) * uu15));
        const V G = V(w0) * (fmadd(V(S(-3)), uFt, m.S) - rS1);
        const V heq = fmadd(V(w0 - S(1)), etamu, phih);
        emit(0, fmadd(om1, g[0], fmadd(omg, geq, gsrcg * G)), fmadd(omh1, h[0], omh * heq));
    }
#pragma unroll
    for (int i = 1; i <= 6; ++i) {
        if (i == 3 || i == 4) continue;          // pairs (1,3) (2,4) (5,7) (6,8)
        const int j = opp_of(i);
        const int cx = cx_of(i), cy = cy_of(i);
        const S w = w_of<S>(i);
        const S c2 = S(cx * cx + cy * cy);
        const V cu = cdot(cx, cy, m.ux, m.uy);
        const V cF = cdot(cx, cy, m.Fx, m.Fy);
        const V cFt = cdot(cx, cy, m.Ftx, m.Fty);
        const V geq_e = V(w) * fmadd(m.rho, fmadd(V(S(4.5)) * cu, cu, uu15), p3);
        const V geq_o = V(S(3) * w) * (m.rho * cu);
        const V G_e = V(w) * fmadd(V(S(9)) * cu, cFt,
                                   fmadd(V(S(-3)), uFt, fmadd(V(S(1.5) * (c2 - S(2) / S(3))), rS1, m.S)));
        const V G_o = V(S(3) * w) * cF;
        const V heq_e = V(w) * etamu;
        const V heq_o = V(S(3) * w) * cdot(cx, cy, phiux, phiuy);
        const V R_o = V(hsc(C.src_h * S(3) * w)) * cdot(cx, cy, ddx, ddy);
        emit(i, fmadd(om1, g[i], fmadd(omg, geq_e + geq_o, gsrcg * (G_e + G_o))),
             fmadd(omh1, h[i], fmadd(omh, heq_e + heq_o, R_o)));
        emit(j, fmadd(om1, g[j], fmadd(omg, geq_e - geq_o, gsrcg * (G_e - G_o))),
             fmadd(omh1, h[j], fmadd(omh, heq_e - heq_o, -R_o)));
    }
}

template <typename V, typename S>
__device__ __forceinline__ void collide_cell(const Consts<S>& C, const Macro<V>& m, V phi, V mu,
                                             V ddx, V ddy, const V g[9], const V h[9],
                                             V gpost[9], V hpost[9]) {
    collide_emit(C, m, phi, mu, ddx, ddy, g, h, [&](int i, V gi, V hi) {
        gpost[i] = gi;
        hpost[i] = hi;
    });
}

// ---------------------------------------------------------------------------
// Asynchronous copies global -> shared by each thread for itself (LDGSTS):
// the data lands in shared memory without passing through registers, and
// cp.async.wait_all makes this thread's copies visible to it.
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                     static_cast<unsigned>(__cvta_generic_to_shared(dst))),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(
                     static_cast<unsigned>(__cvta_generic_to_shared(dst))),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                     static_cast<unsigned>(__cvta_generic_to_shared(dst))),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// ---------------------------------------------------------------------------
// Per-step monitor (optional, a template switch of the step kernels): mass
// sum(phi), kinetic energy sum(rho |u|^2 / 2) and max |u| of the cells each block
// collides, at the time level of the step's input. FP32 forms add phi in a
// float-float pair (TwoSum), so the block sum keeps about 48 bits -- sum(phi)
// stays exact enough to watch its conservation -- at a few FP32 operations a
// cell; the block's result is combined in FP64 and written to its own slot of
// StepArgs::mon (kMonQ doubles), with no atomics, so the sums do not depend on
// timing.
template <typename R> struct MonAcc;
template <> struct MonAcc<double> {
    double m = 0.0, ke = 0.0, u2 = 0.0;
    __device__ __forceinline__ void add(double phi, double lo, double rho, double ux, double uy) {
        m += phi + lo;
        const double uu = ux * ux + uy * uy;
        ke += 0.5 * rho * uu;
        u2 = fmax(u2, uu);
    }
    __device__ __forceinline__ void result(double& mass, double& kin, double& umax2) const {
        mass = m; kin = ke; umax2 = u2;
    }
};
template <> struct MonAcc<float> {
    float mh = 0.f, ml = 0.f, ke = 0.f, u2 = 0.f;
    __device__ __forceinline__ void add(float phi, float lo, float rho, float ux, float uy) {
        float sm, e;
        two_sum(mh, phi, sm, e);
        mh = sm;
        ml += e + lo;
        const float uu = ux * ux + uy * uy;
        ke += 0.5f * rho * uu;
        u2 = fmaxf(u2, uu);
    }
    __device__ __forceinline__ void result(double& mass, double& kin, double& umax2) const {
        mass = double(mh) + double(ml); kin = double(ke); umax2 = double(u2);
    }
};
// Two cells a thread (the paired kernel): the same sums kept per lane of the
// packed FP32 instructions (TwoSum in FADD2), lanes combined in FP64 at the end.
template <> struct MonAcc<F2> {
    F2 mh = F2(0.f), ml = F2(0.f), ke = F2(0.f);
    float u2 = 0.f;
    __device__ __forceinline__ void add(F2 phi, F2 lo, F2 rho, F2 ux, F2 uy) {
        const F2 sm = mh + phi;                      // TwoSum, lane by lane
        const F2 bb = sm - mh;
        const F2 e = (mh - (sm - bb)) + (phi - bb);
        mh = sm;
        ml = ml + (e + lo);
        const F2 uu = fmadd(ux, ux, uy * uy);
        ke = fmadd(F2(0.5f) * rho, uu, ke);
        u2 = fmaxf(u2, fmaxf(uu.v.x, uu.v.y));
    }
    __device__ __forceinline__ void result(double& mass, double& kin, double& umax2) const {
        mass = (double(mh.v.x) + double(ml.v.x)) + (double(mh.v.y) + double(ml.v.y));
        kin = double(ke.v.x) + double(ke.v.y);
        umax2 = double(u2);
    }
};

// Block reduction of the monitor sums; thread 0 writes {sum phi, kinetic
// energy, max |u|^2, non-finite flag} to this block's slot a.mon[item]. The
// instance's record is then formed by a two-level tree without a second launch
// and without many blocks queueing on one counter: the block counts itself in
// its sub-group's counter (sub-group = its position within the instance's items
// modulo kMonSub); the last block of a sub-group adds that sub-group's slots
// (positions s, s + kMonSub, ... in order) into the sub-group's slot and counts
// itself at the instance level; the last of those adds the sub-group slots in
// order and writes the record (max |u|^2 becomes max |u|, plus the non-finite
// flag, the status word and the time level). Every sum has a fixed order, so the
// record does not depend on which blocks finish last.
//
// The group of threads doing this is a whole block (bar 0, grp 0) or one of the
// thread groups of the batched kernel (named barrier `bar`, group `grp` < 4,
// nthr threads, tid its index in the group); item is the work item whose slot
// the group writes, pos its position within its instance's items.
__device__ __forceinline__ void group_sync(int bar, int nthr) {
    if (bar == 0) {   // the whole block (a compile-time 0 wherever a kernel passes it)
        __syncthreads();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nthr) : "memory");
    }
}

// Sums (max for q = 2) of four quantities over a group, fixed tree; result in
// thread 0's v. red: the group's [4][8] shared scratch.
__device__ __forceinline__ void group_reduce4(double v[4], int tid, int nthr, int bar, double (*red)[8]) {
    const int lane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v[0] += __shfl_down_sync(0xffffffffu, v[0], o);
        v[1] += __shfl_down_sync(0xffffffffu, v[1], o);
        v[2] = fmax(v[2], __shfl_down_sync(0xffffffffu, v[2], o));
        v[3] += __shfl_down_sync(0xffffffffu, v[3], o);
    }
    group_sync(bar, nthr);   // red[] may still be read by an earlier use
    if (lane == 0) { red[0][warp] = v[0]; red[1][warp] = v[1]; red[2][warp] = v[2]; red[3][warp] = v[3]; }
    group_sync(bar, nthr);
    if (tid == 0)
        for (int w = 1; w < nwarps; ++w) {
            v[0] += red[0][w];
            v[1] += red[1][w];
            v[2] = fmax(v[2], red[2][w]);
            v[3] += red[3][w];
        }
}

// Atomic add at GPU scope with acquire-release ordering: the caller's earlier
// writes are visible to any thread that sees the new count, and the caller
// sees the writes of every thread whose add came before its own.
__device__ __forceinline__ int atom_add_acq_rel_gpu(int* p, int v) {
    int old;
    asm volatile("atom.add.acq_rel.gpu.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

template <typename R>
__device__ __forceinline__ void mon_block_store(const MonAcc<R>& acc, const StepArgs& a, int inst, int item,
                                                int pos, int tid, int nthr, int bar, int grp) {
    __shared__ double red_all[4][4][8];   // [group][quantity][warp]: up to 8 warps a group
    __shared__ int flag_all[4];
    double (*red)[8] = red_all[grp];
    int& flag = flag_all[grp];
    double v[4];
    acc.result(v[0], v[1], v[2]);
    v[3] = 0.0;
    group_reduce4(v, tid, nthr, bar, red);
    const int* idx = a.mon_csr + a.mon_n + 1;
    const int first = a.mon_csr[inst], items = a.mon_csr[inst + 1] - first;
    const int nsub = items < kMonSub ? items : kMonSub;
    const int s = pos % kMonSub;
    const int in_sub = (items - s + kMonSub - 1) / kMonSub;   // positions s, s + kMonSub, ...
    int* cnt = a.mon_count + (long long)inst * (kMonSub + 1) * kCounterStride;
    if (tid == 0) {
        double* out = a.mon + (long long)item * kMonQ;
        out[0] = v[0];
        out[1] = v[1];
        out[2] = v[2];
        out[3] = (isfinite(v[0]) && isfinite(v[1])) ? 0.0 : 1.0;
        // release: the slot before the count; acquire (for the last): the
        // sub-group's other slots before the reads below, which the barrier
        // orders after this thread's acquire
        flag = atom_add_acq_rel_gpu(cnt + s * kCounterStride, 1) == in_sub - 1;
    }
    group_sync(bar, nthr);
    if (!flag) return;
    // the sub-group's slots, in order
    double w[4] = {0.0, 0.0, 0.0, 0.0};
    for (int j = tid; j < in_sub; j += nthr) {
        const double* p = a.mon_all + (long long)idx[first + s + j * kMonSub] * kMonQ;
        w[0] += __ldcg(p);
        w[1] += __ldcg(p + 1);
        w[2] = fmax(w[2], __ldcg(p + 2));
        w[3] += __ldcg(p + 3);
    }
    group_reduce4(w, tid, nthr, bar, red);
    if (tid == 0) {
        double* sub = a.mon_sub + ((long long)inst * kMonSub + s) * kMonQ;
        sub[0] = w[0];
        sub[1] = w[1];
        sub[2] = w[2];
        sub[3] = w[3];
        cnt[s * kCounterStride] = 0;                      // ready for the next monitored step
        flag = atom_add_acq_rel_gpu(cnt + kMonSub * kCounterStride, 1) == nsub - 1;
    }
    group_sync(bar, nthr);   // (every thread read the first flag before group_reduce4's barriers)
    if (!flag || tid >= 32) return;
    // the instance's record from its sub-group slots: lane q < nsub of the
    // group's first warp loads slot q (the loads in parallel), lane 0 adds them
    // in order q = 0, 1, ...
    double sv[4] = {0.0, 0.0, 0.0, 0.0};
    if (tid < nsub) {
        const double* sb = a.mon_sub + ((long long)inst * kMonSub + tid) * kMonQ;
        sv[0] = __ldcg(sb);
        sv[1] = __ldcg(sb + 1);
        sv[2] = __ldcg(sb + 2);
        sv[3] = __ldcg(sb + 3);
    }
    double m = 0.0, e = 0.0, u = 0.0, f = 0.0;
    for (int q = 0; q < nsub; ++q) {
        const double a0 = __shfl_sync(0xffffffffu, sv[0], q), a1 = __shfl_sync(0xffffffffu, sv[1], q);
        const double a2 = __shfl_sync(0xffffffffu, sv[2], q), a3 = __shfl_sync(0xffffffffu, sv[3], q);
        m += a0;
        e += a1;
        u = fmax(u, a2);
        f += a3;
    }
    if (tid == 0) {
        MonRecord r;
        r.sum_phi = m;
        r.kinetic_energy = e;
        r.max_u = sqrt(u);
        r.nonfinite = f != 0.0 ? 1 : 0;
        r.device_status = *(volatile int*)a.status;
        r.time = a.mon_step + a.time_base[inst];
        a.mon_rec[inst] = r;
        if (a.mon_host) a.mon_host[inst] = r;             // caller's pinned host record, written from here
        cnt[kMonSub * kCounterStride] = 0;
    }
}

// Monitor of every step of a persistent launch (step_kernel_x2_multi with the
// record of each step), the two-level tree of mon_block_store kept per step s
// of the launch: the group reduces its item's sums into slot
// a.mon[(s * a.ndesc + item) * kMonQ] and counts itself in its sub-group's
// counter (sub-group = its position pos within the instance's items modulo
// kMonSub; counters a.mon_count[(s * a.mon_n + inst) * (kMonSub + 1) + ...],
// zeroed before the launch); the last of a sub-group adds the sub-group's slots
// in order into a.mon_sub[((s * a.mon_n + inst) * kMonSub + sub) * kMonQ] and
// counts itself at the instance level; the last of those adds the sub-group
// slots in order and writes the record of step s: into a.mon_host[s * a.mon_n +
// inst] (the caller's pinned host records) and, for the launch's last step,
// a.mon_rec[inst]. Steps of a persistent launch overlap, so this runs while
// other blocks are on later steps; the two levels keep the work of the block
// that finishes a step last short, since its neighbours wait for it.
template <typename R>
__device__ __forceinline__ void mon_step_store(const MonAcc<R>& acc, const StepArgs& a, int inst, int item,
                                               int pos, int tid, int nthr, int bar, int grp, int s) {
    __shared__ double sred_all[4][4][8];
    __shared__ int sflag_all[4];
    double (*red)[8] = sred_all[grp];
    int& flag = sflag_all[grp];
    double v[4];
    acc.result(v[0], v[1], v[2]);
    v[3] = 0.0;
    group_reduce4(v, tid, nthr, bar, red);
    const int* idx = a.mon_csr + a.mon_n + 1;
    const int first = a.mon_csr[inst], items = a.mon_csr[inst + 1] - first;
    const int nsub = items < kMonSub ? items : kMonSub;
    const int sg = pos % kMonSub;
    const int in_sub = (items - sg + kMonSub - 1) / kMonSub;   // positions sg, sg + kMonSub, ...
    const long long si = (long long)s * a.mon_n + inst;
    int* cnt = a.mon_count + si * (kMonSub + 1);
    double* slot = a.mon + (long long)s * a.ndesc * kMonQ;
    if (tid == 0) {
        double* out = slot + (long long)item * kMonQ;
        out[0] = v[0];
        out[1] = v[1];
        out[2] = v[2];
        out[3] = (isfinite(v[0]) && isfinite(v[1])) ? 0.0 : 1.0;
        flag = atom_add_acq_rel_gpu(cnt + sg, 1) == in_sub - 1;
    }
    group_sync(bar, nthr);
    if (!flag) return;
    double w[4] = {0.0, 0.0, 0.0, 0.0};
    for (int j = tid; j < in_sub; j += nthr) {
        const double* p = slot + (long long)idx[first + sg + j * kMonSub] * kMonQ;
        w[0] += __ldcg(p);
        w[1] += __ldcg(p + 1);
        w[2] = fmax(w[2], __ldcg(p + 2));
        w[3] += __ldcg(p + 3);
    }
    group_reduce4(w, tid, nthr, bar, red);
    double* subs = a.mon_sub + si * kMonSub * kMonQ;
    if (tid == 0) {
        double* sub = subs + sg * kMonQ;
        sub[0] = w[0];
        sub[1] = w[1];
        sub[2] = w[2];
        sub[3] = w[3];
        flag = atom_add_acq_rel_gpu(cnt + kMonSub, 1) == nsub - 1;
    }
    group_sync(bar, nthr);   // (every thread read the first flag before group_reduce4's barriers)
    if (!flag || tid >= 32) return;
    // the record from the sub-group slots: lane q < nsub loads slot q, lane 0
    // adds them in order q = 0, 1, ...
    double sv[4] = {0.0, 0.0, 0.0, 0.0};
    if (tid < nsub) {
        sv[0] = __ldcg(subs + tid * kMonQ);
        sv[1] = __ldcg(subs + tid * kMonQ + 1);
        sv[2] = __ldcg(subs + tid * kMonQ + 2);
        sv[3] = __ldcg(subs + tid * kMonQ + 3);
    }
    double m = 0.0, e = 0.0, u = 0.0, f = 0.0;
    for (int q = 0; q < nsub; ++q) {
        m += __shfl_sync(0xffffffffu, sv[0], q);
        e += __shfl_sync(0xffffffffu, sv[1], q);
        u = fmax(u, __shfl_sync(0xffffffffu, sv[2], q));
        f += __shfl_sync(0xffffffffu, sv[3], q);
    }
    if (tid == 0) {
        MonRecord r;
        r.sum_phi = m;
        r.kinetic_energy = e;
        r.max_u = sqrt(u);
        r.nonfinite = f != 0.0 ? 1 : 0;
        r.device_status = *(volatile int*)a.status;
        r.time = a.mon_step + s + a.time_base[inst];
        if (s == a.nsteps - 1) a.mon_rec[inst] = r;
        if (a.mon_host) a.mon_host[si] = r;
    }
}

// ---------------------------------------------------------------------------
// The fused step kernel. Rings in shared memory (slots by row number, powers of
// two so a slot is one AND):
//   phi   [8][TX+4]      rows Y-2 .. Y+2 (and the lead row being written)
//   mu    [4][TX+2]      rows Y-1 .. Y+1
//   p     [4][TX+2]      rows Y-1 .. Y+1 of the previous step's pressure
//   h     [4][P][TX+4]   post-streaming h of rows Y .. Y+3d over the strip and
//                        its 2-column halo (P = 9 planes; conservative forms keep
//                        h_0 as a float pair in the first two planes' room)
// ASYNC (FP32 storage of h and p): each thread copies the h and p values of its
// own columns of the next iteration's lead row (Y + 3d) and p row (Y + 2d) into
// these rings with cp.async right after the first barrier of the iteration, so
// the copies fly during the mu pass and the collision; the next phase A only
// waits for its own copies. Otherwise phase A loads them synchronously.
template <int FORM, int TX>
struct StepSmem {
    using F = Form<FORM>;
    using R = typename F::R;
    static constexpr int PW = TX + 4;   // phi / h ring row: strip + 2-column halo each side
    static constexpr int MW = TX + 2;   // mu / p ring row: strip + 1-column halo
    static constexpr int HPL = F::cons ? 10 : 9;   // R-sized planes of one h slot
    static constexpr size_t elems = 8 * PW + 4 * MW + 4 * MW + 4 * HPL * PW;
    static constexpr size_t bytes = elems * sizeof(R);
};

// Resident blocks per SM the register budget is sized for: FP32 forms 1024/TX
// blocks (64 registers a thread), FP64 384/TX (170 registers; FP64 is bound by
// its arithmetic on GB300, and its shared-memory rings allow few blocks anyway).
template <int FORM, int TX>
struct StepOcc {
    static constexpr int value = (sizeof(typename Form<FORM>::R) == 8 ? 384 : 1024) / TX > 0
                                     ? (sizeof(typename Form<FORM>::R) == 8 ? 384 : 1024) / TX : 1;
};

// The asynchronous variant needs 4- or 8-byte elements for h and p (cp.async).
template <int FORM>
constexpr bool kAsyncOk = sizeof(typename Form<FORM>::R) == 4 && !Form<FORM>::h16;

template <int FORM, int TX, bool ASYNC, bool MON = false>
__global__ void __launch_bounds__(TX, StepOcc<FORM, TX>::value) step_kernel(const StepArgs a) {
    using F = Form<FORM>;
    using R = typename F::R;
    using AT = typename F::AT;
    using SM = StepSmem<FORM, TX>;
    static_assert(!ASYNC || kAsyncOk<FORM>, "asynchronous copies need 4-byte h and p");
    constexpr int PW = SM::PW, MW = SM::MW, HPL = SM::HPL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* phiR = reinterpret_cast<R*>(smem_raw);   // [8][PW]
    R* muR = phiR + 8 * PW;                      // [4][MW]
    R* pR = muR + 4 * MW;                        // [4][MW]
    R* hR = pR + 4 * MW;                         // [4][HPL][PW]

    const WorkItem wk = a.work[blockIdx.x];
    Consts<R> C;
    C.load(a.inst[wk.inst]);
    const int nx = C.nx, ny = C.ny, walls = C.walls;
    const int x0 = wk.x0, d = wk.dir;
    const int w = min(TX, nx - x0);
    const int tid = threadIdx.x;
    const int base = (int)C.base;       // cell indices fit in 32 bits (checked on the host)
    const long long S = a.S;

    PopIO<F> io;
    io.hin = static_cast<const typename F::HT*>(a.h_in);
    io.hout = static_cast<typename F::HT*>(a.h_out);
    io.h0in = static_cast<const float2*>(a.h0_in);
    io.h0out = static_cast<float2*>(a.h0_out);
    io.gin = static_cast<const typename F::GT*>(a.g_in);
    io.gout = static_cast<typename F::GT*>(a.g_out);
    io.S = S; io.hs = C.hs; io.ihs = C.ihs; io.gs = C.gs; io.igs = C.igs;
    const AT* p_in = static_cast<const AT*>(a.p_in);
    AT* p_out = static_cast<AT*>(a.p_out);
    AT* phiu = static_cast<AT*>(a.phiu);
    MonAcc<R> mon;

    auto wrapx = [nx](int x) { return x < 0 ? x + nx : (x >= nx ? x - nx : x); };
    auto rowg = [ny, walls](int y) { return walls ? y : (y < 0 ? y + ny : (y >= ny ? y - ny : y)); };
    auto ghost = [ny, walls](int y) { return walls && (y < 0 || y >= ny); };
    auto mirror = [ny](int y) { return y < 0 ? -1 - y : 2 * ny - 1 - y; };
    auto rowoff = [&](int y) { return base + rowg(y) * nx; };
    // h slot of row y: plane i (i >= 1 for conservative forms) at hplane(y, i)[s],
    // conservative h_0 pair at hpair(y)[s]
    auto hslot = [&](int y) { return hR + ((y + 64) & 3) * HPL * PW; };
    auto hplane = [&](int y, int i) { return hslot(y) + (F::cons ? i + 1 : i) * PW; };
    auto hpair = [&](int y) { return reinterpret_cast<float2*>(hslot(y)); };

    // Per-thread columns, fixed for the whole march.
    const bool lead0 = tid < w + 4, lead1 = tid + TX < w + 4;      // phi / h columns x0-2+s
    const int lc0 = lead0 ? wrapx(x0 - 2 + tid) : 0;
    const int lc1 = lead1 ? wrapx(x0 - 2 + tid + TX) : 0;
    const bool mid0 = tid < w + 2, mid1 = tid + TX < w + 2;       // mu / p columns x0-1+s
    const int pc0 = mid0 ? wrapx(x0 - 1 + tid) : 0;
    const int pc1 = mid1 ? wrapx(x0 - 1 + tid + TX) : 0;
    const bool act = tid < w;                                     // collision column X
    const int X = x0 + tid;
    const int colm = act ? wrapx(X - 1) : 0, colp = act ? wrapx(X + 1) : 0;

    // phi (and its low part) of column s from h values already in the slot of row L
    auto phi_from_slot = [&](int L, int s) {
        R* prow = phiR + ((L + 64) & 7) * PW;
        if constexpr (F::cons) {
            R s8 = R(0);
#pragma unroll
            for (int i = 1; i < 9; ++i) s8 += hplane(L, i)[s];
            float2* pr = hpair(L);
            const float2 h0 = pr[s];
            float sm, e, hi, lo;
            two_sum(h0.x, s8, sm, e);
            fast_two_sum(sm, e + h0.y, hi, lo);
            prow[s] = hi;
            pr[s].y = lo;                      // low part of phi, read by the collision
        } else {
            R phi = hplane(L, 0)[s];
#pragma unroll
            for (int i = 1; i < 9; ++i) phi += hplane(L, i)[s];
            prow[s] = phi;
        }
    };
    auto ghost_row = [&](int L) {   // mirror ghost row next to a wall (reading Q7)
        R* prow = phiR + ((L + 64) & 7) * PW;
        const R* src = phiR + ((mirror(L) + 64) & 7) * PW;
        if (lead0) prow[tid] = src[tid];
        if (lead1) prow[tid + TX] = src[tid + TX];
    };
    // A (synchronous). phi of row L over columns x0-2 .. x0+w+1; h kept in the slot.
    auto lead_row = [&](int L) {
        if (ghost(L)) { ghost_row(L); return; }
        const int ro = rowoff(L);
        R* prow = phiR + ((L + 64) & 7) * PW;
        auto column = [&](int s, int col) {
            R hv[9], lo;
            prow[s] = io.phi_of(ro + col, hv, lo);          // Eq. 18
            if constexpr (F::cons) {
                hpair(L)[s] = make_float2(hv[0], lo);
#pragma unroll
                for (int i = 1; i < 9; ++i) hplane(L, i)[s] = hv[i];
            } else {
#pragma unroll
                for (int i = 0; i < 9; ++i) hplane(L, i)[s] = hv[i];
            }
        };
        if (lead0) column(tid, lc0);
        if (lead1) column(tid + TX, lc1);
    };
    // p of the previous step, row M, columns x0-1 .. x0+w (mirror ghost at walls).
    auto p_row = [&](int M) {
        const AT* src = p_in + base + (ghost(M) ? mirror(M) : rowg(M)) * nx;
        R* dst = pR + ((M + 64) & 3) * MW;
        if (mid0) dst[tid] = R(src[pc0]);
        if (mid1) dst[tid + TX] = R(src[pc1]);
    };
    // Asynchronous copies of this thread's columns of lead row L and p row M.
    auto prefetch = [&](int L, int M) {
        if constexpr (ASYNC) {
            if (!ghost(L)) {
                const int ro = rowoff(L);
                auto column = [&](int s, int col) {
                    const int cc = ro + col;
                    if constexpr (F::cons) {
                        cp_async8(&hpair(L)[s], io.h0in + cc);
#pragma unroll
                        for (int i = 1; i < 9; ++i) cp_async4(&hplane(L, i)[s], io.hin + io.hoff(i) + cc);
                    } else {
#pragma unroll
                        for (int i = 0; i < 9; ++i) cp_async4(&hplane(L, i)[s], io.hin + io.hoff(i) + cc);
                    }
                };
                if (lead0) column(tid, lc0);
                if (lead1) column(tid + TX, lc1);
            }
            const AT* src = p_in + base + (ghost(M) ? mirror(M) : rowg(M)) * nx;
            R* dst = pR + ((M + 64) & 3) * MW;
            if (mid0) cp_async4(&dst[tid], src + pc0);
            if (mid1) cp_async4(&dst[tid + TX], src + pc1);
            cp_async_commit();
        }
    };
    // A (asynchronous). phi of row L from the values this thread copied itself.
    auto lead_row_async = [&](int L) {
        cp_async_wait_all();
        if (ghost(L)) { ghost_row(L); return; }
        if (lead0) phi_from_slot(L, tid);
        if (lead1) phi_from_slot(L, tid + TX);
    };
    // B. mu of row M (Eq. 8 with the Laplacian of Eq. 30b), columns x0-1 .. x0+w.
    auto mu_row = [&](int M) {
        R* mrow = muR + ((M + 64) & 3) * MW;
        if (ghost(M)) {
            const R* src = muR + ((mirror(M) + 64) & 3) * MW;
            if (mid0) mrow[tid] = src[tid];
            if (mid1) mrow[tid + TX] = src[tid + TX];
            return;
        }
        const R* r0 = phiR + ((M - 1 + 64) & 7) * PW;
        const R* r1 = phiR + ((M + 64) & 7) * PW;
        const R* r2 = phiR + ((M + 1 + 64) & 7) * PW;
        auto column = [&](int s) {
            Nbr<R> n;
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
                n.z[0][dx] = r0[s + dx];
                n.z[1][dx] = r1[s + dx];
                n.z[2][dx] = r2[s + dx];
            }
            mrow[s] = chem_pot(C, n.z[1][1], n.lap());
        };
        if (mid0) column(tid);
        if (mid1) column(tid + TX);
    };
    // C. collision and push-streaming of row Y (g, phi u of the previous step loaded early).
    auto collide_row = [&](int Y, const R (&g)[9], R pux, R puy) {
        if (!act) return;
        const int rY = rowoff(Y);
        const int c = rY + X;
        Nbr<R> nphi, nmu, np;
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
            const R* pr = phiR + ((Y + dy - 1 + 64) & 7) * PW + tid + 1;
            const R* mr = muR + ((Y + dy - 1 + 64) & 3) * MW + tid;
            const R* qr = pR + ((Y + dy - 1 + 64) & 3) * MW + tid;
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
                nphi.z[dy][dx] = pr[dx];
                nmu.z[dy][dx] = mr[dx];
                np.z[dy][dx] = qr[dx];
            }
        }
        const R phi = nphi.z[1][1], mu = nmu.z[1][1];
        R gphix, gphiy, gmux, gmuy, gpx, gpy;
        nphi.grad(gphix, gphiy);
        nmu.grad(gmux, gmuy);
        np.grad(gpx, gpy);
        const R lapmu = nmu.lap();
        R h[9];
        if constexpr (F::cons) {
            h[0] = hpair(Y)[tid + 2].y;        // low part of phi
#pragma unroll
            for (int i = 1; i < 9; ++i) h[i] = hplane(Y, i)[tid + 2];
        } else {
#pragma unroll
            for (int i = 0; i < 9; ++i) h[i] = hplane(Y, i)[tid + 2];
        }

        const Macro<R> m = macroscopic(C, g, phi, mu, gphix, gphiy, gmux, gmuy, lapmu, gpx, gpy);
        const R phiux = phi * m.ux, phiuy = phi * m.uy;
        if constexpr (MON) mon.add(phi, F::cons ? h[0] : R(0), m.rho, m.ux, m.uy);
        R gpost[9], hpost[9];
        collide_cell(C, m, phi, mu, phiux - pux, phiuy - puy, g, h, gpost, hpost);

        float2 h0c = make_float2(0.f, 0.f);
        if constexpr (F::cons) {
            // h_0 absorbs the storage rounding of h_1..h_8: the stored populations
            // of this cell still sum to phi (collision conserves phi: sum h^eq = phi,
            // sum R_i = 0), so rounding cannot change sum(phi).
            R rest = R(0);
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                hpost[i] = io.round_h(hpost[i]);
                rest += hpost[i];
            }
            h0c = io.conservative_h0(phi, h[0] /* low part of phi */, rest);
        }
        // Push-streaming: population i moves to x + c_i; into a wall it comes back
        // reversed at x (halfway bounce-back, Sec. 4.3). Wall rows are uniform per row.
        const bool bot = walls && Y == 0, top = walls && Y == ny - 1;
        const int rDn = bot ? 0 : rowoff(Y - 1);
        const int rUp = top ? 0 : rowoff(Y + 1);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int cyi = cy_of(i), cxi = cx_of(i);
            const int col = cxi < 0 ? colm : (cxi > 0 ? colp : X);
            int dst = (cyi == 0 ? rY : (cyi > 0 ? rUp : rDn)) + col;
            int k = i;
            if ((cyi > 0 && top) || (cyi < 0 && bot)) {
                dst = c;
                k = opp_of(i);
            }
            if constexpr (F::cons) {
                if (i == 0) io.store_h0(dst, h0c);
                else io.store_h(k, dst, hpost[i]);
            } else {
                io.store_h(k, dst, hpost[i]);
            }
            io.store_g(k, dst, gpost[i]);
        }
        phiu[c] = AT(phiux);
        phiu[S + c] = AT(phiuy);
        p_out[c] = AT(m.p);
    };

    const int Y0 = wk.ystart;
    // Prologue: phi rows Y0-2d .. Y0+d, mu rows Y0-d .. Y0, p rows Y0-d .. Y0.
    // Rows inside the domain first: a ghost row (beyond a wall, on either side
    // of Y0) copies its mirror row, which must exist by then.
    for (int pass = 0; pass < 2; ++pass)
        for (int k = 1; k >= -2; --k)
            if (ghost(Y0 + k * d) == (pass == 1)) lead_row(Y0 + k * d);
    p_row(Y0 - d);
    p_row(Y0);
    __syncthreads();
    // the slot of row Y0 - 2d (read only above) takes the first lead row
    if constexpr (ASYNC) prefetch(Y0 + 2 * d, Y0 + d);
    mu_row(Y0);
    mu_row(Y0 - d);
    __syncthreads();
    for (int k = 0; k < wk.nrows; ++k) {
        const int Y = Y0 + k * d;
        // g and phi*u of the collision row, loaded before the barriers so the
        // loads overlap phases A and B
        R g[9];
        R pux = R(0), puy = R(0);
        if (act) {
            const int c = rowoff(Y) + X;
#pragma unroll
            for (int i = 0; i < 9; ++i) g[i] = io.load_g(i, c);
            pux = R(phiu[c]);
            puy = R(phiu[S + c]);
        }
        if constexpr (ASYNC) {
            lead_row_async(Y + 2 * d);
        } else {
            lead_row(Y + 2 * d);
            p_row(Y + d);
        }
        __syncthreads();
        // Every thread is past the collision of row Y - d: the h slot of row Y - d
        // and the p slot of row Y - 2d are free for the next iteration's rows.
        if constexpr (ASYNC) {
            if (k + 1 < wk.nrows) prefetch(Y + 3 * d, Y + 2 * d);
        }
        mu_row(Y + d);
        __syncthreads();
        collide_row(Y, g, pux, puy);
    }
    if constexpr (MON) mon_block_store(mon, a, wk.inst, blockIdx.x, wk.pad, threadIdx.x, TX, 0, 0);
}

}  // namespace lbm
