// lbm_d3q15.cu -- the phase-field model of Sec. 3 on the three-dimensional D3Q15
// lattice of Sec. 2.2 (weights 2/9, 1/9 x 6, 1/72 x 8; c_s^2 = 1/3; d = 3 in
// Eq. 34 and in the printed G_0).
//
// One time step is three kernels over the cells of an instance, one thread a
// cell (x fastest):
//   phi3_kernel     phi = sum_i h_i (Eq. 18) into a scratch plane (conservative
//                   form: the float pair hi + lo, the low part in its own plane);
//   mu3_kernel      mu of Eq. 8 with the 14-neighbour Laplacian of Eq. 30b;
//   collide3_kernel the macroscopic stage (Eq. 30 gradients of phi, mu and the
//                   previous step's p; forces, u of Eq. 27a, S, tau_g, Eq. 28 /
//                   29), the collisions of Eqs. 24 and 10 and push-streaming of
//                   both sets (x and z periodic; halfway bounce-back at walls
//                   normal to y; the stencils see a wall as a mirror, reading Q7).
// phi and mu go through global memory (L2-resident for the neighbour reads): the
// 2-D kernels' strip march keeps them on chip instead, but a 3-D march would
// need rings of whole planes of 15 populations. Storage forms: FP64, FP32, and
// FP32 with the two-float h_0 (the conservative form of the 2-D path).
#include <cstdint>

#include "lbm.h"
#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {
namespace d3 {

constexpr int Q = 15;
// D3Q15 velocities in the order printed in Sec. 2.2.
__host__ __device__ constexpr int cx(int i) {
    return i == 1 ? 1 : i == 4 ? -1 : (i == 7 || i == 8 || i == 9 || i == 14) ? 1 : (i >= 10 && i <= 13) ? -1 : 0;
}
__host__ __device__ constexpr int cy(int i) {
    return i == 2 ? 1 : i == 5 ? -1 : (i == 7 || i == 8 || i == 10 || i == 13) ? 1 : (i == 9 || i == 11 || i == 12 || i == 14) ? -1 : 0;
}
__host__ __device__ constexpr int cz(int i) {
    return i == 3 ? 1 : i == 6 ? -1 : (i == 7 || i == 9 || i == 10 || i == 12) ? 1 : (i == 8 || i == 11 || i == 13 || i == 14) ? -1 : 0;
}
__host__ __device__ constexpr double w(int i) { return i == 0 ? 2.0 / 9.0 : (i <= 6 ? 1.0 / 9.0 : 1.0 / 72.0); }
__host__ __device__ constexpr int opp(int i) {
    for (int k = 0; k < Q; ++k)
        if (cx(k) == -cx(i) && cy(k) == -cy(i) && cz(k) == -cz(i)) return k;
    return 0;
}
static_assert(cx(7) == 1 && cy(7) == 1 && cz(7) == 1 && cx(14) == 1 && cy(14) == -1 && cz(14) == -1, "D3Q15 order");
static_assert(opp(1) == 4 && opp(7) == 11 && opp(14) == 10, "D3Q15 opposites");

// storage of the three 3-D forms: R is both the arithmetic and the storage type
template <int FORM> struct F3;
template <> struct F3<0> { using R = double; static constexpr bool cons = false; };
template <> struct F3<1> { using R = float; static constexpr bool cons = false; };
template <> struct F3<4> { using R = float; static constexpr bool cons = true; };

struct Geo {
    int nx, ny, nz, walls;
    long long base;
    __device__ __forceinline__ void load(const DevInst& P) {
        nx = P.nx; ny = P.ny; nz = P.nz; walls = P.walls; base = P.base;
    }
    __device__ __forceinline__ int wrap(int v, int n) const { return v < 0 ? v + n : (v >= n ? v - n : v); }
    // neighbour of (x, y, z) in direction i for the stencils (mirror at walls)
    __device__ __forceinline__ long long nbr(int x, int y, int z, int i) const {
        const int xx = wrap(x + cx(i), nx), zz = wrap(z + cz(i), nz);
        int yy = y + cy(i);
        if (walls) yy = yy < 0 ? -1 - yy : (yy >= ny ? 2 * ny - 1 - yy : yy);
        else yy = wrap(yy, ny);
        return base + ((long long)zz * ny + yy) * nx + xx;
    }
};

template <typename R>
struct Grad3 { R x, y, z, lap; };

// Eq. 30a / 30b over the 14 neighbours of a field stored in global memory.
template <typename R, typename T>
__device__ __forceinline__ Grad3<R> stencil(const T* f, const Geo& G, int x, int y, int z, R center) {
    Grad3<R> d{R(0), R(0), R(0), R(0)};
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const R v = R(f[G.nbr(x, y, z, i)]);
        const R wv = R(w(i)) * v;
        if (cx(i)) d.x += cx(i) > 0 ? wv : -wv;
        if (cy(i)) d.y += cy(i) > 0 ? wv : -wv;
        if (cz(i)) d.z += cz(i) > 0 ? wv : -wv;
        d.lap += R(w(i)) * (v - center);
    }
    d.x *= R(3); d.y *= R(3); d.z *= R(3);   // 1 / c_s^2
    d.lap *= R(6);                            // 2 / c_s^2
    return d;
}

struct Args {
    StepArgs s;     // h_in/out, h0_in/out, g_in/out, phiu (3 planes), p_in/out, S, inst, status
    void* phi;      // scratch plane: phi (R)
    void* mu;       // scratch plane: mu (R)
    float* philo;   // scratch plane: low part of phi (conservative form)
    int instance;
    int ncells;
};

template <int FORM>
__device__ __forceinline__ void cell_xyz(const Geo& G, int cell, int& x, int& y, int& z) {
    x = cell % G.nx;
    const int t = cell / G.nx;
    y = t % G.ny;
    z = t / G.ny;
}

// phi = sum_i h_i (Eq. 18).
template <int FORM>
__global__ void __launch_bounds__(256) phi3_kernel(const Args a) {
    using R = typename F3<FORM>::R;
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= a.ncells) return;
    const DevInst& P = a.s.inst[a.instance];
    const long long c = P.base + cell;
    const R* h = static_cast<const R*>(a.s.h_in);
    R* phi = static_cast<R*>(a.phi);
    if constexpr (F3<FORM>::cons) {
        float rest = 0.f;
#pragma unroll
        for (int i = 1; i < Q; ++i) rest += h[(long long)(i - 1) * a.s.S + c];
        const float2 h0 = static_cast<const float2*>(a.s.h0_in)[c];
        float s, e, hi, lo;
        two_sum(h0.x, rest, s, e);
        fast_two_sum(s, e + h0.y, hi, lo);
        phi[c] = hi;
        a.philo[c] = lo;
    } else {
        R sum = h[c];
#pragma unroll
        for (int i = 1; i < Q; ++i) sum += h[(long long)i * a.s.S + c];
        phi[c] = sum;
    }
}

// mu of Eq. 8 from the phi plane.
template <int FORM>
__global__ void __launch_bounds__(256) mu3_kernel(const Args a) {
    using R = typename F3<FORM>::R;
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= a.ncells) return;
    const DevInst& P = a.s.inst[a.instance];
    Geo G;
    G.load(P);
    Consts<R> C;
    C.load(P);
    int x, y, z;
    cell_xyz<FORM>(G, cell, x, y, z);
    const R* phi = static_cast<const R*>(a.phi);
    const long long c = P.base + cell;
    const R ph = phi[c];
    const Grad3<R> d = stencil<R>(phi, G, x, y, z, ph);
    static_cast<R*>(a.mu)[c] = chem_pot(C, ph, d.lap);
}

// Macroscopic stage of one cell (steps 1-6 of the time step in 3-D).
template <typename R>
struct Macro3 {
    R rho, u[3], F[3], Ft[3], S, S1, tgm, inv_tau_g, p;
};

template <typename R>
__device__ __forceinline__ Macro3<R> macroscopic3(const Consts<R>& C, const R g[Q], R phi, R mu,
                                                  const Grad3<R>& dphi, const Grad3<R>& dmu,
                                                  const Grad3<R>& dp) {
    Macro3<R> m;
    m.rho = fma(phi, C.drho, C.rho_B);                                   // Eq. 3aa
    const R dr[3] = {C.drho * dphi.x, C.drho * dphi.y, C.drho * dphi.z};
    m.S1 = C.qim ? -C.gammaM * dmu.lap : R(0);                           // Sec. 3.2.1
    if (C.sforce == 0) {
        m.F[0] = mu * dphi.x; m.F[1] = mu * dphi.y; m.F[2] = mu * dphi.z;
    } else {
        m.F[0] = -phi * dmu.x; m.F[1] = -phi * dmu.y; m.F[2] = -phi * dmu.z;
    }
    m.F[0] += C.force_x;
    m.F[1] += C.force_y - (m.rho - C.rho_A) * C.gravity;                 // buoyancy, Sec. 4.4
    R j[3] = {R(0), R(0), R(0)};
    R sum_g = R(0);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        if (cx(i)) j[0] += cx(i) > 0 ? g[i] : -g[i];
        if (cy(i)) j[1] += cy(i) > 0 ? g[i] : -g[i];
        if (cz(i)) j[2] += cz(i) > 0 ? g[i] : -g[i];
        sum_g += g[i];
    }
    const R inv_rho = rcp(m.rho);
#pragma unroll
    for (int a = 0; a < 3; ++a) m.u[a] = fma(R(0.5), m.F[a], j[a]) * inv_rho;   // Eq. 27a
    m.S = m.u[0] * dr[0] + m.u[1] * dr[1] + m.u[2] * dr[2] + m.rho * m.S1;
    if (C.uniform_nu) {
        m.tgm = C.tgm0;
        m.inv_tau_g = C.inv_tau_g0;
    } else {
        R nu;
        if (C.visc == 0) nu = rcp(fma(phi, C.inv_nu_A - C.inv_nu_B, C.inv_nu_B));
        else nu = step_pick(phi, C.mu_A, C.mu_B) * inv_rho;
        m.tgm = R(3) * nu;
        m.inv_tau_g = rcp(m.tgm + R(0.5));
    }
    const R dpv[3] = {dp.x, dp.y, dp.z};
#pragma unroll
    for (int a = 0; a < 3; ++a) m.Ft[a] = m.F[a] - dpv[a] + dr[a] * (R(1) / R(3));   // F~
    const R w0 = R(w(0));
    R G0 = R(0);
    if (C.pscheme == 0) {   // printed simplification, d = 3: w0 [(2/3) rho S1 - 3 u.(F - grad p)]
        const R uFp = m.u[0] * (m.F[0] - dpv[0]) + m.u[1] * (m.F[1] - dpv[1]) + m.u[2] * (m.F[2] - dpv[2]);
        G0 = w0 * (R(2.0 / 3.0) * m.rho * m.S1 - R(3) * uFp);
    } else if (C.pscheme == 1) {   // Eq. 34 at i = 0
        const R uFt = m.u[0] * m.Ft[0] + m.u[1] * m.Ft[1] + m.u[2] * m.Ft[2];
        G0 = w0 * (m.S - R(3) * uFt - m.rho * m.S1);
    }
    const R uu = m.u[0] * m.u[0] + m.u[1] * m.u[1] + m.u[2] * m.u[2];
    // Eq. 28 (29): c_s^2 / (1 - w0) = 3/7; s_0(u) = -w0 u.u / (2 c_s^2) = -u.u / 3
    m.p = R(3.0 / 7.0) * (sum_g + R(0.5) * m.S - m.rho * uu * R(1.0 / 3.0) + m.tgm * G0);
    return m;
}

// Collision and push-streaming of one cell, given phi (and its low part in the
// conservative form), mu and the three stencils; loads the cell's own g, h and
// the previous step's phi u, stores both sets at their destinations, phi u and p.
template <int FORM>
__device__ __forceinline__ void collide_cell3(const Args& a, const DevInst& P, const Geo& Gm,
                                              const Consts<typename F3<FORM>::R>& C, int x, int y, int z,
                                              typename F3<FORM>::R phi, typename F3<FORM>::R phi_lo,
                                              typename F3<FORM>::R mu,
                                              const Grad3<typename F3<FORM>::R>& dphi,
                                              const Grad3<typename F3<FORM>::R>& dmu,
                                              const Grad3<typename F3<FORM>::R>& dp) {
    using R = typename F3<FORM>::R;
    constexpr bool cons = F3<FORM>::cons;
    const long long c = P.base + ((long long)z * Gm.ny + y) * Gm.nx + x;
    const long long S = a.s.S;
    const R* hin = static_cast<const R*>(a.s.h_in);
    const R* gin = static_cast<const R*>(a.s.g_in);
    R* hout = static_cast<R*>(a.s.h_out);
    R* gout = static_cast<R*>(a.s.g_out);
    R* phiu = static_cast<R*>(a.s.phiu);

    R g[Q], h[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) g[i] = gin[(long long)i * S + c];
    if constexpr (cons) {
#pragma unroll
        for (int i = 1; i < Q; ++i) h[i] = hin[(long long)(i - 1) * S + c];
        h[0] = R(0);   // unused: the conservative h_0 is formed from phi below
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) h[i] = hin[(long long)i * S + c];
    }
    const Macro3<R> m = macroscopic3(C, g, phi, mu, dphi, dmu, dp);
    const R pu[3] = {phi * m.u[0], phi * m.u[1], phi * m.u[2]};
    const R dpu[3] = {pu[0] - phiu[c], pu[1] - phiu[S + c], pu[2] - phiu[2 * S + c]};
    const R uu = m.u[0] * m.u[0] + m.u[1] * m.u[1] + m.u[2] * m.u[2];
    const R uFt = m.u[0] * m.Ft[0] + m.u[1] * m.Ft[1] + m.u[2] * m.Ft[2];
    const R ig = m.inv_tau_g, srcg = R(1) - R(0.5) * ig;
    const R ih = C.inv_tau_h, srch = C.src_h;
    const R em = C.eta * mu;
    const bool bot = Gm.walls && y == 0, top = Gm.walls && y == Gm.ny - 1;
    // destination coordinates for offsets -1, 0, +1 (cell indices fit 32 bits)
    const int xs[3] = {Gm.wrap(x - 1, Gm.nx), x, Gm.wrap(x + 1, Gm.nx)};
    const int ys[3] = {Gm.walls ? y - 1 : Gm.wrap(y - 1, Gm.ny), y, Gm.walls ? y + 1 : Gm.wrap(y + 1, Gm.ny)};
    const int zs[3] = {Gm.wrap(z - 1, Gm.nz), z, Gm.wrap(z + 1, Gm.nz)};
    float rest = 0.f;   // conservative form: sum of the stored h_1 .. h_14
    // push-streaming of direction i: to x + c_i, or back into this cell reversed at a wall
    auto emit = [&](int i, R gpost, R hpost) {
        long long dst;
        int k = i;
        if ((cy(i) > 0 && top) || (cy(i) < 0 && bot)) {
            dst = c;
            k = opp(i);
        } else {
            dst = P.base + ((zs[cz(i) + 1] * Gm.ny + ys[cy(i) + 1]) * Gm.nx + xs[cx(i) + 1]);
        }
        gout[(long long)k * S + dst] = gpost;
        if constexpr (cons) {
            if (i == 0) return;   // h_0 after the loop, from phi and the stored others
            rest += hpost;
            hout[(long long)(k - 1) * S + dst] = hpost;
        } else {
            hout[(long long)k * S + dst] = hpost;
        }
    };
    {   // rest direction: s_0 = -w_0 u.u / (2 c_s^2), G_0 and h_0^eq of Eqs. 33, 34, 11
        const R w0 = R(w(0));
        const R s0 = w0 * (-R(1.5) * uu);
        const R geq = R(3) * m.p * (w0 - R(1)) + m.rho * s0;                                    // Eq. 33
        const R G0 = w0 * (m.S - R(3) * uFt - m.rho * m.S1);                                    // Eq. 34
        const R heq = phi + (w0 - R(1)) * em;                                                   // Eq. 11
        emit(0, g[0] - (g[0] - geq) * ig + srcg * G0, h[0] - (h[0] - heq) * ih);
    }
    // the moving directions in opposite pairs (i, opp(i)): c_opp = -c_i, so each
    // of s_i, G_i, h_i^eq and R_i splits into a part even in c (shared) and a
    // part odd in c (sign flipped)
    constexpr int kPair[7] = {1, 2, 3, 7, 8, 9, 10};
#pragma unroll
    for (int q = 0; q < 7; ++q) {
        const int i = kPair[q], j = opp(i);
        const R wi = R(w(i));
        const R cu = R(cx(i)) * m.u[0] + R(cy(i)) * m.u[1] + R(cz(i)) * m.u[2];
        const R cF = R(cx(i)) * m.F[0] + R(cy(i)) * m.F[1] + R(cz(i)) * m.F[2];
        const R cFt = R(cx(i)) * m.Ft[0] + R(cy(i)) * m.Ft[1] + R(cz(i)) * m.Ft[2];
        const R c2 = R(cx(i) * cx(i) + cy(i) * cy(i) + cz(i) * cz(i));
        // Eq. 33 (rho_0 = 0: g_0 is stored shifted by rho_0): w_i p / c_s^2 + rho s_i
        const R geq_e = R(3) * m.p * wi + m.rho * (wi * (R(4.5) * cu * cu - R(1.5) * uu));
        const R geq_o = m.rho * (wi * (R(3) * cu));
        // Eq. 34: w_i [S + c.F / c_s^2 + (2 (c.u)(c.Ft) - 2 c_s^2 u.Ft) / (2 c_s^4)
        //              + (|c|^2 - d c_s^2)(2/d) rho c_s^2 S1 / (2 c_s^4)], d = 3
        const R G_e = wi * (m.S + R(9) * cu * cFt - R(3) * uFt + (c2 - R(1)) * m.rho * m.S1);
        const R G_o = wi * (R(3) * cF);
        // Eq. 11 and Eq. 14
        const R heq_e = wi * em;
        const R heq_o = R(3) * wi * (R(cx(i)) * pu[0] + R(cy(i)) * pu[1] + R(cz(i)) * pu[2]);
        const R R_o = srch * R(3) * wi * (R(cx(i)) * dpu[0] + R(cy(i)) * dpu[1] + R(cz(i)) * dpu[2]);
        emit(i, g[i] - (g[i] - (geq_e + geq_o)) * ig + srcg * (G_e + G_o),                       // Eq. 24
             h[i] - (h[i] - (heq_e + heq_o)) * ih + R_o);                                         // Eq. 10
        emit(j, g[j] - (g[j] - (geq_e - geq_o)) * ig + srcg * (G_e - G_o),
             h[j] - (h[j] - (heq_e - heq_o)) * ih - R_o);
    }
    if constexpr (cons) {
        // h_0 = phi - sum of the stored h_1..h_14, as a float pair: sum(phi) is conserved
        float s, e, hi, lo;
        two_sum(phi, -rest, s, e);
        fast_two_sum(s, e + phi_lo, hi, lo);
        static_cast<float2*>(a.s.h0_out)[c] = make_float2(hi, lo);
    }
    phiu[c] = pu[0];
    phiu[S + c] = pu[1];
    phiu[2 * S + c] = pu[2];
    static_cast<R*>(a.s.p_out)[c] = m.p;
}

// Unfused step, third kernel (phi and mu from the scratch planes); also the
// step of LBM_PIPELINE_PLAIN. 4 blocks of 256 threads a SM (64 registers):
// measured on the 128 x 256 x 128 bubble, FP32 6.5k -> 8.5k MLUPS against the
// unbounded 108 registers (2 blocks).
template <int FORM>
__global__ void __launch_bounds__(256, 4) collide3_kernel(const Args a) {
    using R = typename F3<FORM>::R;
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= a.ncells) return;
    const DevInst& P = a.s.inst[a.instance];
    Geo Gm;
    Gm.load(P);
    Consts<R> C;
    C.load(P);
    int x, y, z;
    cell_xyz<FORM>(Gm, cell, x, y, z);
    const long long c = P.base + cell;
    const R* phi_f = static_cast<const R*>(a.phi);
    const R* mu_f = static_cast<const R*>(a.mu);
    const R* p_in = static_cast<const R*>(a.s.p_in);
    const R phi = phi_f[c], mu = mu_f[c];
    const R phi_lo = F3<FORM>::cons ? R(a.philo[c]) : R(0);
    const Grad3<R> dphi = stencil<R>(phi_f, Gm, x, y, z, phi);
    const Grad3<R> dmu = stencil<R>(mu_f, Gm, x, y, z, mu);
    const Grad3<R> dp = stencil<R>(p_in, Gm, x, y, z, p_in[c]);
    collide_cell3<FORM>(a, P, Gm, C, x, y, z, phi, phi_lo, mu, dphi, dmu, dp);
}

// ---------------------------------------------------------------------------
// Fused step: a block owns a TX x TY tile of (x, y) columns of one instance and
// marches in z over a run of planes (direction d = +-1), as the 2-D kernels march
// rows. Per collision plane Z:
//   (A) phi of plane Z + 2d over the tile and a 2-cell halo, from the 15 h of
//       each cell (global memory), into a ring of 8 planes in shared memory;
//       p of plane Z + 2d (previous step) over the tile and a 1-cell halo;
//   (B) mu of plane Z + d over the tile and a 1-cell halo, from the phi ring;
//   (C) the collision of plane Z with the phi, mu and p stencils from shared
//       memory (collide_cell3 reloads the cell's own h, now in L2).
// Two barriers a plane; (A) of the next plane writes ring slots that (C) of this
// plane does not read. Halo cells beyond a wall are the mirror cells (Q7).
template <int FORM, int TX, int TY>
struct March3 {
    using R = typename F3<FORM>::R;
    static constexpr int PX = TX + 4, PY = TY + 4;   // phi tile + 2-cell halo
    static constexpr int MX = TX + 2, MY = TY + 2;   // mu / p tile + 1-cell halo
    static constexpr int NT = TX * TY;
    // dynamic shared memory: phi ring (8 planes), mu ring (4), p ring (8), low
    // parts of phi (4 planes of the tile, conservative form)
    static constexpr size_t PHI = 0;
    static constexpr size_t MU = PHI + sizeof(R) * 8 * PX * PY;
    static constexpr size_t PP = MU + sizeof(R) * 4 * MX * MY;
    static constexpr size_t LO = PP + sizeof(R) * 8 * MX * MY;
    static constexpr size_t bytes = LO + (F3<FORM>::cons ? sizeof(float) * 4 * NT : 0);
};

// resident blocks the register budget is sized for: FP32 3 (85 registers), FP64 2
template <int FORM> constexpr int kMarchOcc = FORM == 0 ? 2 : 3;

template <int FORM, int TX, int TY>
__global__ void __launch_bounds__(TX * TY, kMarchOcc<FORM>) march3_kernel(const Args a,
                                                                          const WorkItem* __restrict__ work) {
    using R = typename F3<FORM>::R;
    using L = March3<FORM, TX, TY>;
    constexpr int PX = L::PX, PY = L::PY, MX = L::MX, MY = L::MY, NT = L::NT;
    extern __shared__ __align__(16) unsigned char smem3[];
    R (*phiR)[PY * PX] = reinterpret_cast<R (*)[PY * PX]>(smem3 + L::PHI);
    R (*muR)[MY * MX] = reinterpret_cast<R (*)[MY * MX]>(smem3 + L::MU);
    R (*pR)[MY * MX] = reinterpret_cast<R (*)[MY * MX]>(smem3 + L::PP);
    float (*loR)[NT] = reinterpret_cast<float (*)[NT]>(smem3 + L::LO);   // conservative form only

    const WorkItem wk = work[blockIdx.x];
    const DevInst& P = a.s.inst[wk.inst];
    Geo Gm;
    Gm.load(P);
    Consts<R> C;
    C.load(P);
    const int x0 = wk.x0, y0 = wk.pad, d = wk.dir;
    const int wx = min(TX, Gm.nx - x0), wy = min(TY, Gm.ny - y0);
    const int t = threadIdx.x;
    const long long S = a.s.S;
    const R* hin = static_cast<const R*>(a.s.h_in);
    const R* p_in = static_cast<const R*>(a.s.p_in);

    auto ymap = [&](int y) {   // halo row -> stored row (mirror at walls, wrap otherwise)
        if (Gm.walls) return y < 0 ? -1 - y : (y >= Gm.ny ? 2 * Gm.ny - 1 - y : y);
        return Gm.wrap(y, Gm.ny);
    };
    const int plane = Gm.nx * Gm.ny;   // cells of one z plane (instance cells fit 32 bits)

    // Loop-invariant per-thread work of the plane phases: each thread handles at
    // most two phi cells (tile + 2-cell halo) and two mu / p cells (tile + 1-cell
    // halo); their in-plane global offsets and ring indices are fixed for the run.
    constexpr int NA = (PX * PY + NT - 1) / NT, NB = (MX * MY + NT - 1) / NT;
    static_assert(NA <= 2 && NB <= 2, "tile too small for two cells a thread");
    int a_yx[NA], a_sm[NA], a_lo[NA];
    int b_yx[NB], b_sm[NB], b_phi[NB];
#pragma unroll
    for (int j = 0; j < NA; ++j) {
        const int k = t + j * NT;
        const int hx = k % PX - 2, hy = k / PX - 2;
        const bool ok = k < PX * PY && hx < wx + 2 && hy < wy + 2;
        a_sm[j] = ok ? k : -1;
        a_yx[j] = ok ? ymap(y0 + hy) * Gm.nx + Gm.wrap(x0 + hx, Gm.nx) : 0;
        a_lo[j] = (ok && hx >= 0 && hx < TX && hy >= 0 && hy < TY) ? hy * TX + hx : -1;
    }
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        const int k = t + j * NT;
        const int hx = k % MX - 1, hy = k / MX - 1;
        const bool ok = k < MX * MY && hx < wx + 1 && hy < wy + 1;
        b_sm[j] = ok ? k : -1;
        b_yx[j] = ok ? ymap(y0 + hy) * Gm.nx + Gm.wrap(x0 + hx, Gm.nx) : 0;
        b_phi[j] = (hy + 2) * PX + hx + 2;
    }
    auto slot8 = [](int z) { return (z + 1024) & 7; };
    auto slot4 = [](int z) { return (z + 1024) & 3; };

    // (A) phi of plane Zl (tile + 2-cell halo), low parts of the tile cells.
    auto phi_plane = [&](int Zl) {
        const long long zb = P.base + (long long)Gm.wrap(Zl, Gm.nz) * plane;
        R* dst = phiR[slot8(Zl)];
#pragma unroll
        for (int j = 0; j < NA; ++j) {
            if (a_sm[j] < 0) continue;
            const long long c = zb + a_yx[j];
            if constexpr (F3<FORM>::cons) {
                float rest = 0.f;
#pragma unroll
                for (int i = 1; i < Q; ++i) rest += hin[(long long)(i - 1) * S + c];
                const float2 h0 = static_cast<const float2*>(a.s.h0_in)[c];
                float sm, e, hi, lo;
                two_sum(h0.x, rest, sm, e);
                fast_two_sum(sm, e + h0.y, hi, lo);
                dst[a_sm[j]] = hi;
                if (a_lo[j] >= 0) loR[slot4(Zl)][a_lo[j]] = lo;
            } else {
                R sum = hin[c];
#pragma unroll
                for (int i = 1; i < Q; ++i) sum += hin[(long long)i * S + c];
                dst[a_sm[j]] = sum;
            }
        }
    };
    // p of plane Zp (tile + 1-cell halo); 8 planes: the next plane's (A) writes
    // p of Z + 3d while lagging threads may still read p of Z - d in (C)
    auto p_plane = [&](int Zp) {
        const long long zb = P.base + (long long)Gm.wrap(Zp, Gm.nz) * plane;
        R* dst = pR[slot8(Zp)];
#pragma unroll
        for (int j = 0; j < NB; ++j)
            if (b_sm[j] >= 0) dst[b_sm[j]] = p_in[zb + b_yx[j]];
    };
    // 14-neighbour Eq. 30 stencil over three ring planes (z - 1, z, z + 1) at a
    // ring index; the neighbour offsets are compile-time
    auto stencil_ring = [&](const R* zm, const R* z0, const R* zp, int at, int rowlen) {
        Grad3<R> g{R(0), R(0), R(0), R(0)};
        const R c0 = z0[at];
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const R* pl = cz(i) < 0 ? zm : (cz(i) > 0 ? zp : z0);
            const R v = pl[at + cy(i) * rowlen + cx(i)];
            const R wv = R(w(i)) * v;
            if (cx(i)) g.x += cx(i) > 0 ? wv : -wv;
            if (cy(i)) g.y += cy(i) > 0 ? wv : -wv;
            if (cz(i)) g.z += cz(i) > 0 ? wv : -wv;
            g.lap += R(w(i)) * (v - c0);
        }
        g.x *= R(3); g.y *= R(3); g.z *= R(3); g.lap *= R(6);
        return g;
    };
    // (B) mu of plane Zm (tile + 1-cell halo)
    auto mu_plane = [&](int Zm) {
        R* dst = muR[slot4(Zm)];
        const R* f0 = phiR[slot8(Zm - 1)];
        const R* f1 = phiR[slot8(Zm)];
        const R* f2 = phiR[slot8(Zm + 1)];
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            if (b_sm[j] < 0) continue;
            const int at = b_phi[j];
            const R c0 = f1[at];
            R lap = R(0);
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                const R* pl = cz(i) < 0 ? f0 : (cz(i) > 0 ? f2 : f1);
                lap += R(w(i)) * (pl[at + cy(i) * PX + cx(i)] - c0);
            }
            dst[b_sm[j]] = chem_pot(C, c0, R(6) * lap);
        }
    };

    const int Z0 = wk.ystart;
    // prologue: phi of planes Z0-2d .. Z0+d, mu of Z0-d and Z0, p of Z0-d .. Z0+d
    for (int k = -2; k <= 1; ++k) phi_plane(Z0 + k * d);
    p_plane(Z0 - d);
    p_plane(Z0);
    p_plane(Z0 + d);
    __syncthreads();
    mu_plane(Z0 - d);
    mu_plane(Z0);
    __syncthreads();
    const int tx = t % TX, ty = t / TX;
    const bool act = tx < wx && ty < wy;
    const int at_phi = (ty + 2) * PX + tx + 2, at_m = (ty + 1) * MX + tx + 1;
    for (int k = 0; k < wk.nrows; ++k) {
        const int Z = Z0 + k * d;
        phi_plane(Z + 2 * d);       // (A)
        p_plane(Z + 2 * d);
        __syncthreads();
        mu_plane(Z + d);            // (B)
        __syncthreads();
        if (act) {                  // (C)
            const R* f1 = phiR[slot8(Z)];
            const R phi = f1[at_phi];
            const R phi_lo = F3<FORM>::cons ? R(loR[slot4(Z)][ty * TX + tx]) : R(0);
            const R mu = muR[slot4(Z)][at_m];
            const Grad3<R> dphi = stencil_ring(phiR[slot8(Z - 1)], f1, phiR[slot8(Z + 1)], at_phi, PX);
            const Grad3<R> dmu = stencil_ring(muR[slot4(Z - 1)], muR[slot4(Z)], muR[slot4(Z + 1)], at_m, MX);
            const Grad3<R> dp = stencil_ring(pR[slot8(Z - 1)], pR[slot8(Z)], pR[slot8(Z + 1)], at_m, MX);
            collide_cell3<FORM>(a, P, Gm, C, x0 + tx, y0 + ty, Gm.wrap(Z, Gm.nz), phi, phi_lo, mu, dphi, dmu,
                                dp);
        }
    }
}

// Initial state (reading Q6): h = h^eq(phi0, mu0, u = 0), g = 0 (g^eq at p = 0,
// u = 0, shifted by rho_0), phi u = 0, p = 0. phi0: the instance's cells in FP64.
template <int FORM>
__global__ void __launch_bounds__(256) init3_kernel(const Args a, const double* __restrict__ phi0) {
    using R = typename F3<FORM>::R;
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= a.ncells) return;
    const DevInst& P = a.s.inst[a.instance];
    Geo G;
    G.load(P);
    G.base = 0;   // neighbours index phi0 from 0
    Consts<double> C;
    C.load(P);
    int x, y, z;
    cell_xyz<FORM>(G, cell, x, y, z);
    const double ph = phi0[cell];
    const Grad3<double> d = stencil<double>(phi0, G, x, y, z, ph);
    const double em = C.eta * chem_pot(C, ph, d.lap);
    const long long c = P.base + cell, S = a.s.S;
    R* h = static_cast<R*>(a.s.h_out);
    R* g = static_cast<R*>(a.s.g_out);
    R* phiu = static_cast<R*>(a.s.phiu);
    double rest = 0.0;
    for (int i = 1; i < Q; ++i) {
        const R hi = R(w(i) * em);
        rest += double(hi);
        h[(long long)(F3<FORM>::cons ? i - 1 : i) * S + c] = hi;
    }
    const double h0 = ph + (w(0) - 1.0) * em;
    if constexpr (F3<FORM>::cons) {
        // the pair holds phi0 - (stored h_1..h_14) to about 48 bits
        const double r = ph - rest;
        const float hi = float(r);
        static_cast<float2*>(a.s.h0_out)[c] = make_float2(hi, float(r - double(hi)));
    } else {
        h[c] = R(h0);
    }
    for (int i = 0; i < Q; ++i) g[(long long)i * S + c] = R(0);
    phiu[c] = R(0); phiu[S + c] = R(0); phiu[2 * S + c] = R(0);
    static_cast<R*>(a.s.p_out)[c] = R(0);
    static_cast<R*>(const_cast<void*>(a.s.p_in))[c] = R(0);
}

// Fields of one instance (same arithmetic as the collision's macroscopic stage):
// bits of mask in the order phi, ux, uy, p, rho, mu, P (Sec. 4.2), uz.
template <int FORM>
__global__ void __launch_bounds__(256) fields3_kernel(const Args a, unsigned mask, double* __restrict__ out,
                                                      double* __restrict__ partials) {
    using R = typename F3<FORM>::R;
    constexpr int kQ = kDiagQuantities;
    double acc[kQ];
#pragma unroll
    for (int q = 0; q < kQ; ++q) acc[q] = 0.0;
    const DevInst& P = a.s.inst[a.instance];
    Geo Gm;
    Gm.load(P);
    Consts<R> C;
    C.load(P);
    const long long S = a.s.S;
    const R* gin = static_cast<const R*>(a.s.g_in);
    const R* hin = static_cast<const R*>(a.s.h_in);
    const R* phi_f = static_cast<const R*>(a.phi);
    const R* mu_f = static_cast<const R*>(a.mu);
    const R* p_in = static_cast<const R*>(a.s.p_in);
    for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < a.ncells; cell += gridDim.x * blockDim.x) {
        int x, y, z;
        cell_xyz<FORM>(Gm, cell, x, y, z);
        const long long c = P.base + cell;
        R g[Q];
        bool fin = true;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            g[i] = gin[(long long)i * S + c];
            fin = fin && isfinite(g[i]);
        }
#pragma unroll
        for (int i = 0; i < (F3<FORM>::cons ? Q - 1 : Q); ++i) fin = fin && isfinite(hin[(long long)i * S + c]);
        const R phi = phi_f[c], mu = mu_f[c];
        const Grad3<R> dphi = stencil<R>(phi_f, Gm, x, y, z, phi);
        const Grad3<R> dmu = stencil<R>(mu_f, Gm, x, y, z, mu);
        const Grad3<R> dp = stencil<R>(p_in, Gm, x, y, z, p_in[c]);
        const Macro3<R> m = macroscopic3(C, g, phi, mu, dphi, dmu, dp);
        double ph = double(phi);
        if constexpr (F3<FORM>::cons) ph += double(a.philo[c]);
        // P = p_0 - kappa phi lap(phi) + kappa |grad phi|^2 / 2 + p (Sec. 4.2)
        const double b = double(C.beta), k = double(C.kappa);
        const double psi = b * ph * ph * (ph - 1.0) * (ph - 1.0);
        const double dpsi = 2.0 * b * ph * (ph - 1.0) * (2.0 * ph - 1.0);
        const double g2 = double(dphi.x) * double(dphi.x) + double(dphi.y) * double(dphi.y) +
                          double(dphi.z) * double(dphi.z);
        const double Pl = ph * dpsi - psi - k * ph * double(dphi.lap) + 0.5 * k * g2 + double(m.p);
        if (out) {
            const double v[8] = {ph, double(m.u[0]), double(m.u[1]), double(m.p), double(m.rho),
                                 double(mu), Pl, double(m.u[2])};
            int slot = 0;
            for (int bit = 0; bit < 8; ++bit)
                if (mask & (1u << bit)) out[(long long)(slot++) * a.ncells + cell] = v[bit];
        }
        if (partials) {
            const double rho = double(m.rho);
            const double uu = double(m.u[0]) * double(m.u[0]) + double(m.u[1]) * double(m.u[1]) +
                              double(m.u[2]) * double(m.u[2]);
            acc[0] += ph;
            acc[1] += rho;
            acc[2] += 0.5 * rho * uu;
            acc[3] = fmax(acc[3], sqrt(uu));
            acc[4] += ph * x;
            acc[5] += ph * y;
            acc[6] += (1.0 - ph) * x;
            acc[7] += (1.0 - ph) * y;
            if (ph > 1.0 - 1e-3) { acc[8] += Pl; acc[9] += 1.0; }
            if (ph < 1e-3) { acc[10] += Pl; acc[11] += 1.0; }
            if (!fin) acc[12] += 1.0;
            acc[13] += 1.0 - ph;
        }
    }
    if (!partials) return;
    __shared__ double red[kQ][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
        double v = acc[q];
        for (int o = 16; o > 0; o >>= 1) {
            const double t = __shfl_down_sync(0xffffffffu, v, o);
            v = q == 3 ? fmax(v, t) : v + t;
        }
        if (lane == 0) red[q][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < kQ) {
        const int q = threadIdx.x;
        double v = red[q][0];
        for (int k2 = 1; k2 < (int)(blockDim.x >> 5); ++k2) v = q == 3 ? fmax(v, red[q][k2]) : v + red[q][k2];
        partials[blockIdx.x * kQ + q] = v;
    }
}

// Fixed-order final sum of the per-block partials (one block).
__global__ void __launch_bounds__(256) diag3_final(const double* __restrict__ partials, int nblocks,
                                                   double* __restrict__ result) {
    constexpr int kQ = kDiagQuantities;
    const int t = threadIdx.x;
    double acc[kQ];
#pragma unroll
    for (int q = 0; q < kQ; ++q) acc[q] = 0.0;
    for (int b = t; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            const double v = partials[b * kQ + q];
            acc[q] = q == 3 ? fmax(acc[q], v) : acc[q] + v;
        }
    __shared__ double red[kQ][8];
    const int lane = t & 31, warp = t >> 5;
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
        double v = acc[q];
        for (int o = 16; o > 0; o >>= 1) {
            const double u = __shfl_down_sync(0xffffffffu, v, o);
            v = q == 3 ? fmax(v, u) : v + u;
        }
        if (lane == 0) red[q][warp] = v;
    }
    __syncthreads();
    if (t < kQ) {
        double v = red[t][0];
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) v = t == 3 ? fmax(v, red[t][k]) : v + red[t][k];
        result[t] = v;
    }
}

// Populations of one instance in FP64 (h_0 of the conservative form = hi + lo).
template <int FORM>
__global__ void __launch_bounds__(256) populations3_kernel(const Args a, double* __restrict__ out_h,
                                                           double* __restrict__ out_g) {
    using R = typename F3<FORM>::R;
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= a.ncells) return;
    const DevInst& P = a.s.inst[a.instance];
    const long long c = P.base + cell, S = a.s.S, n = a.ncells;
    const R* h = static_cast<const R*>(a.s.h_in);
    const R* g = static_cast<const R*>(a.s.g_in);
    for (int i = 0; i < Q; ++i) {
        out_g[i * n + cell] = double(g[(long long)i * S + c]);
        if (F3<FORM>::cons) {
            if (i == 0) {
                const float2 p = static_cast<const float2*>(a.s.h0_in)[c];
                out_h[cell] = double(p.x) + double(p.y);
            } else {
                out_h[i * n + cell] = double(h[(long long)(i - 1) * S + c]);
            }
        } else {
            out_h[i * n + cell] = double(h[(long long)i * S + c]);
        }
    }
}

int blocks_for(int n) { return (n + 255) / 256; }

template <typename Fn>
cudaError_t by_form3(int form, Fn&& fn) {
    switch (form) {
        case 0: return fn(std::integral_constant<int, 0>{});
        case 1: return fn(std::integral_constant<int, 1>{});
        case 4: return fn(std::integral_constant<int, 4>{});
        default: return cudaErrorInvalidValue;
    }
}

Args make_args(const StepArgs& s, const D3Scratch& x, int instance, int ncells) {
    Args a;
    a.s = s;
    a.phi = x.phi;
    a.mu = x.mu;
    a.philo = x.philo;
    a.instance = instance;
    a.ncells = ncells;
    return a;
}

}  // namespace d3

bool d3_form_ok(int form) { return form == 0 || form == 1 || form == 4; }

cudaError_t launch_phi_mu3(int form, const StepArgs& s, const D3Scratch& x, int instance, int ncells,
                           cudaStream_t st) {
    const d3::Args a = d3::make_args(s, x, instance, ncells);
    return d3::by_form3(form, [&](auto F) {
        constexpr int FORM = decltype(F)::value;
        d3::phi3_kernel<FORM><<<d3::blocks_for(ncells), 256, 0, st>>>(a);
        d3::mu3_kernel<FORM><<<d3::blocks_for(ncells), 256, 0, st>>>(a);
        return cudaGetLastError();
    });
}

// tile of the fused march: 32 x 8 columns
constexpr int kMarchTX = 32, kMarchTY = 8;

void march3_tile(int* tx, int* ty) {
    *tx = kMarchTX;
    *ty = kMarchTY;
}

cudaError_t prepare_march3(int form) {
    return d3::by_form3(form, [&](auto F) {
        constexpr int FORM = decltype(F)::value;
        return cudaFuncSetAttribute(d3::march3_kernel<FORM, kMarchTX, kMarchTY>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)d3::March3<FORM, kMarchTX, kMarchTY>::bytes);
    });
}

int march3_occupancy(int form) {
    int n = 0;
    d3::by_form3(form, [&](auto F) {
        constexpr int FORM = decltype(F)::value;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, d3::march3_kernel<FORM, kMarchTX, kMarchTY>,
                                                             kMarchTX * kMarchTY,
                                                             d3::March3<FORM, kMarchTX, kMarchTY>::bytes);
    });
    return n;
}

cudaError_t launch_march3(int form, const StepArgs& s, const D3Scratch& x, const WorkItem* work, int nwork,
                          cudaStream_t st) {
    if (nwork <= 0) return cudaSuccess;
    const d3::Args a = d3::make_args(s, x, 0, 0);
    return d3::by_form3(form, [&](auto F) {
        constexpr int FORM = decltype(F)::value;
        d3::march3_kernel<FORM, kMarchTX, kMarchTY>
            <<<nwork, kMarchTX * kMarchTY, d3::March3<FORM, kMarchTX, kMarchTY>::bytes, st>>>(a, work);
        return cudaGetLastError();
    });
}

cudaError_t launch_step3(int form, const StepArgs& s, const D3Scratch& x, int instance, int ncells,
                         cudaStream_t st) {
    cudaError_t e = launch_phi_mu3(form, s, x, instance, ncells, st);
    if (e != cudaSuccess) return e;
    const d3::Args a = d3::make_args(s, x, instance, ncells);
    return d3::by_form3(form, [&](auto F) {
        d3::collide3_kernel<decltype(F)::value><<<d3::blocks_for(ncells), 256, 0, st>>>(a);
        return cudaGetLastError();
    });
}

cudaError_t launch_init3(int form, const StepArgs& s, const D3Scratch& x, int instance, int ncells,
                         const double* phi0, cudaStream_t st) {
    const d3::Args a = d3::make_args(s, x, instance, ncells);
    return d3::by_form3(form, [&](auto F) {
        d3::init3_kernel<decltype(F)::value><<<d3::blocks_for(ncells), 256, 0, st>>>(a, phi0);
        return cudaGetLastError();
    });
}

cudaError_t launch_fields3(int form, const StepArgs& s, const D3Scratch& x, int instance, int ncells,
                           unsigned mask, double* out, double* partials, double* result, cudaStream_t st) {
    cudaError_t e = launch_phi_mu3(form, s, x, instance, ncells, st);
    if (e != cudaSuccess) return e;
    const d3::Args a = d3::make_args(s, x, instance, ncells);
    const int nb = partials ? kDiagBlocks : d3::blocks_for(ncells);
    e = d3::by_form3(form, [&](auto F) {
        d3::fields3_kernel<decltype(F)::value><<<nb, 256, 0, st>>>(a, mask, out, partials);
        return cudaGetLastError();
    });
    if (e != cudaSuccess || !partials) return e;
    d3::diag3_final<<<1, 256, 0, st>>>(partials, kDiagBlocks, result);
    return cudaGetLastError();
}

cudaError_t launch_populations3(int form, const StepArgs& s, const D3Scratch& x, int instance, int ncells,
                                double* out_h, double* out_g, cudaStream_t st) {
    const d3::Args a = d3::make_args(s, x, instance, ncells);
    return d3::by_form3(form, [&](auto F) {
        d3::populations3_kernel<decltype(F)::value><<<d3::blocks_for(ncells), 256, 0, st>>>(a, out_h, out_g);
        return cudaGetLastError();
    });
}

}  // namespace lbm
