// lbm_sp.cu -- the single-phase models of Sec. 2.3 on the D2Q9 lattice: the
// generalized lattice Boltzmann model with a mass source, in the forms of
// Remarks 3, 1 and 2, and the explicit D_i G_i scheme of Remark 4.
//
// Remark 3 (model LBM_SP_INCOMPRESSIBLE_SOURCE): rho~ = rho_0 and a constant
// density (rho = 1), the incompressible Navier-Stokes equations with a mass
// source (div u = S) and a uniform body force. One kernel a step: the cell's
// populations and source give u (Eq. 27a) and p (Eq. 28 with G_0), the
// equilibrium (Eq. 25 with rho~ = rho_0, rho = 1; g_0 stored shifted by rho_0)
// and the force term
//   G_i = w_i { S + c_i.F / c_s^2 + (c_i c_i - c_s^2 I):(u F + F u + Q S I) / (2 c_s^4) },
//   Q = (2/d) c_s^2 - xi / (tau_g - 1/2),
// then BGK (Eq. 24) and push-streaming (x periodic; y periodic or halfway
// bounce-back walls). Storage and arithmetic in FP64 or FP32.
//
// Remark 1 (LBM_SP_NEARLY_INCOMPRESSIBLE; rho~ = rho, p = rho c_s^2): rho =
// sum g + S/2 (Eq. 27aa), u = (sum c g + F/2) / rho, g^eq = rho (w_i + s_i(u))
// (Eq. 29bb), G_i with (u F + F u - u u S + Q div(u) I) and Q = (2/d) rho c_s^2 -
// xi / (tau_g - 1/2); div u by Eq. 30a from a plane of u (mirror at walls), so
// a step is two kernels (rho and u, then the collision). The populations are
// stored as g_i - w_i (their rest state at rho = 1), so that FP32 storage keeps
// the small deviations that carry the flow: rho = 1 + sum(g - w) + S/2.
//
// Remark 2 (LBM_SP_HE_INCOMPRESSIBLE): the same two kernels with g in units of
// pressure (g^eq = w_i p + p_0 s_i(u), Eq. 29bd; p_0 S_1 and p_0 F_1), stored as
// g_i - w_i p_0.
//
// Remark 4 (scheme LBM_SP_SCHEME_REMARK4): the Remark 3 model with a
// velocity-dependent force F(u) = F_0 - (lambda + beta |u|) u, evolved with the
// explicit D_i G_i (unshifted f, u = sum c f). A first kernel writes u and
// F(u); the second rebuilds G_i at the destination x + c_i from its u, F(u) and
// S, and G_i(x, t - 1) from u and F at t - 1 (four planes kept instead of the
// nine planes of G).
//
// FP32 with nx even runs kernels with two horizontally adjacent cells a thread
// in packed FP32 instructions. The collisions of Remarks 1 and 2 and of the
// two-cell Remark 4 kernel take opposite directions in pairs (the parts of s_i
// and G_i even in c shared, the odd parts sign-flipped).
#include <cmath>
#include <cstring>
#include <string>

#include "lbm.h"
#include "lbm_device.cuh"   // lbm::F2, two cells' FP32 values in packed instructions

namespace {

using lbm::F2;
__device__ __forceinline__ F2& operator+=(F2& a, F2 b) { return a = a + b; }
__device__ __forceinline__ F2& operator*=(F2& a, F2 b) { return a = a * b; }
// 1/x and sqrt(x), correctly rounded per lane, so one-cell and two-cell kernels agree
template <typename R> __device__ __forceinline__ R sp_inv(R x) { return R(1) / x; }
__device__ __forceinline__ F2 sp_inv(F2 x) { return F2(1.f / x.v.x, 1.f / x.v.y); }
template <typename R> __device__ __forceinline__ R sp_sqrt(R x) { return sqrt(x); }
__device__ __forceinline__ F2 sp_sqrt(F2 x) { return F2(sqrtf(x.v.x), sqrtf(x.v.y)); }

// Loads and stores of cell pairs (x, x + 1), x even: one 8-byte access.
__device__ __forceinline__ F2 ld2(const float* p) { return F2(*reinterpret_cast<const float2*>(p)); }
__device__ __forceinline__ void st2(float* p, F2 v) { *reinterpret_cast<float2*>(p) = v.v; }
// A row of a plane around the pair: columns x - 2 .. x + 3 as three pairs
// (wrapping in x; nx even). at(dx) is the pair of columns (x + dx, x + 1 + dx).
struct Row2 {
    float2 l, m, r;
    __device__ __forceinline__ Row2(const float* row, int x, int nx) {
        l = *reinterpret_cast<const float2*>(row + (x == 0 ? nx - 2 : x - 2));
        m = *reinterpret_cast<const float2*>(row + x);
        r = *reinterpret_cast<const float2*>(row + (x + 2 == nx ? 0 : x + 2));
    }
    __device__ __forceinline__ F2 at(int dx) const {
        return dx < 0 ? F2(l.y, m.x) : (dx > 0 ? F2(m.y, r.x) : F2(m));
    }
};

constexpr int kQ = 9;
__host__ __device__ constexpr int sx(int i) { return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0); }
__host__ __device__ constexpr int sy(int i) { return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0); }
__host__ __device__ constexpr double sw(int i) { return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0); }
__host__ __device__ constexpr int sopp(int i) { return i == 0 ? 0 : (i <= 4 ? (i + 1) % 4 + 1 : (i - 5 + 2) % 4 + 5); }
static_assert(sopp(1) == 3 && sopp(2) == 4 && sopp(5) == 7 && sopp(6) == 8 && sopp(8) == 6, "D2Q9 opposites");
// one direction of each opposite pair (1, 2, 5, 6; their opposites 3, 4, 7, 8)
__host__ __device__ constexpr int pair2(int q) { return q == 0 ? 1 : q == 1 ? 2 : q == 2 ? 5 : 6; }

// Push-streaming of direction i of a pair (x, x + 1), x even (32-bit offsets:
// the context checks 9 nx ny < 2^31): with bounce, back
// into the pair as the opposite direction (halfway wall); else to row yrow,
// columns x + c_x and x + 1 + c_x (wrapped). c_x = 0 keeps the pair together.
__device__ __forceinline__ void sp_store2(float* __restrict__ gout, int N, int c, int x, int yrow, int nx,
                                          bool bounce, int i, F2 v) {
    if (bounce) {
        st2(gout + sopp(i) * N + c, v);
    } else if (sx(i) == 0) {
        st2(gout + i * N + yrow * nx + x, v);
    } else {
        const int row = i * N + yrow * nx;
        gout[row + (sx(i) < 0 ? (x == 0 ? nx - 1 : x - 1) : x + 1)] = v.v.x;
        gout[row + (sx(i) < 0 ? x : (x + 2 == nx ? 0 : x + 2))] = v.v.y;
    }
}

struct SpConst {
    int nx, ny, walls;
    double inv_tau, src, tgm, Qc, fx, fy;   // 1/tau_g, 1 - 1/(2 tau_g), tau_g - 1/2, Q, F
    double dl, dq;                          // drag of the Remark 4 scheme: F(u) = F - (dl + dq |u|) u
    double p0;                              // Remark 2: the constant p_0
    // derived on the host, so that FP32 kernels do no FP64 arithmetic on them
    double tau, Qd0;                        // tau_g; Q - (2/d) c_s^2 (the part of Q without the density)
    double hp0, ip0, hp0fx, hp0fy;          // p_0 / 2, 1 / p_0, p_0 F_1 / 2
};

template <typename R>
struct SpCell { R ux, uy, p; };

// u (Eq. 27a, rho = 1), G_i (Remark 3) and p (Eq. 28) of one cell
template <typename R>
__device__ __forceinline__ SpCell<R> sp_moments(const SpConst& K, const R g[kQ], R S, R G[kQ]) {
    SpCell<R> m;
    R jx = R(0), jy = R(0), rest = R(0);
#pragma unroll
    for (int i = 1; i < kQ; ++i) {
        if (sx(i)) jx += sx(i) > 0 ? g[i] : -g[i];
        if (sy(i)) jy += sy(i) > 0 ? g[i] : -g[i];
        rest += g[i];
    }
    const R fx = R(K.fx), fy = R(K.fy);
    m.ux = jx + R(0.5) * fx;
    m.uy = jy + R(0.5) * fy;
    const R uF = m.ux * fx + m.uy * fy, uu = m.ux * m.ux + m.uy * m.uy;
    const R QS = R(K.Qc) * S;
    // (c c - c_s^2 I):(u F + F u + Q S I) / (2 c_s^4) = 9 (c.u)(c.F) - 3 u.F + 4.5 (|c|^2 - 2/3) Q S;
    // for opposite directions the part even in c is shared and c.F / c_s^2 flips sign
    G[0] = R(sw(0)) * (S - R(3) * uF + R(4.5) * (-R(2.0 / 3.0)) * QS);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = pair2(q), j = sopp(i);
        const R cu = R(sx(i)) * m.ux + R(sy(i)) * m.uy, cF = R(sx(i)) * fx + R(sy(i)) * fy;
        const R c2 = R(sx(i) * sx(i) + sy(i) * sy(i));
        const R e = R(sw(i)) * (S + R(9) * cu * cF - R(3) * uF + R(4.5) * (c2 - R(2.0 / 3.0)) * QS);
        const R o = R(sw(i)) * (R(3) * cF);
        G[i] = e + o;
        G[j] = e - o;
    }
    // Eq. 28: c_s^2 / (1 - w_0) = 3/5; s_0(u) = -w_0 u.u / (2 c_s^2) = -(2/3) u.u
    m.p = R(0.6) * (rest + R(0.5) * S - R(2.0 / 3.0) * uu + R(K.tgm) * G[0]);
    return m;
}

template <typename R>
__global__ void __launch_bounds__(256) sp_step_kernel(const R* __restrict__ gin, R* __restrict__ gout,
                                                      const R* __restrict__ src, long long N, SpConst K) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int x = (int)(c % K.nx), y = (int)(c / K.nx);
    R g[kQ], G[kQ];
#pragma unroll
    for (int i = 0; i < kQ; ++i) g[i] = gin[i * N + c];
    const R S = src[c];
    const SpCell<R> m = sp_moments(K, g, S, G);
    const R uu = m.ux * m.ux + m.uy * m.uy;
    const R ig = R(K.inv_tau), sg = R(K.src);
    const bool bot = K.walls && y == 0, top = K.walls && y == K.ny - 1;
    const int xs[3] = {x == 0 ? K.nx - 1 : x - 1, x, x == K.nx - 1 ? 0 : x + 1};
    const int ys[3] = {K.walls ? y - 1 : (y == 0 ? K.ny - 1 : y - 1), y,
                       K.walls ? y + 1 : (y == K.ny - 1 ? 0 : y + 1)};
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
        const R cu = R(sx(i)) * m.ux + R(sy(i)) * m.uy;
        const R si = R(sw(i)) * (R(3) * cu + R(4.5) * cu * cu - R(1.5) * uu);
        const R geq = i == 0 ? R(3) * m.p * (R(sw(0)) - R(1)) + si : R(3) * m.p * R(sw(i)) + si;
        const R post = g[i] - (g[i] - geq) * ig + sg * G[i];
        long long dst;
        int k = i;
        if ((sy(i) > 0 && top) || (sy(i) < 0 && bot)) {
            dst = c;
            k = sopp(i);
        } else {
            dst = (long long)ys[sy(i) + 1] * K.nx + xs[sx(i) + 1];
        }
        gout[k * N + dst] = post;
    }
}

// FP32 step of Remark 3 with two horizontally adjacent cells (x, x + 1), x
// even, per thread, computed together in packed FP32 instructions (F2): the
// loads, the S read and the stores of directions with c_x = 0 are 8-byte
// pairs; directions with c_x != 0 split into two 4-byte stores. nx even.
__global__ void __launch_bounds__(256, 4) sp_step_x2_kernel(const float* __restrict__ gin, float* __restrict__ gout,
                                                         const float* __restrict__ src, int N, SpConst K) {
    const int c = 2 * (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (c >= N) return;
    const int x = (int)(c % K.nx), y = (int)(c / K.nx);
    F2 g[kQ], G[kQ];
#pragma unroll
    for (int i = 0; i < kQ; ++i) g[i] = F2(*reinterpret_cast<const float2*>(gin + i * N + c));
    const F2 S(*reinterpret_cast<const float2*>(src + c));
    const SpCell<F2> m = sp_moments(K, g, S, G);
    const F2 uu = m.ux * m.ux + m.uy * m.uy;
    const F2 ig = F2(float(K.inv_tau)), sg = F2(float(K.src));
    const bool bot = K.walls && y == 0, top = K.walls && y == K.ny - 1;
    const int ys[3] = {K.walls ? y - 1 : (y == 0 ? K.ny - 1 : y - 1), y,
                       K.walls ? y + 1 : (y == K.ny - 1 ? 0 : y + 1)};
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
        const F2 cu = float(sx(i)) * m.ux + float(sy(i)) * m.uy;
        const F2 si = float(sw(i)) * (F2(3.f) * cu + F2(4.5f) * cu * cu - F2(1.5f) * uu);
        const F2 geq = i == 0 ? F2(3.f) * m.p * F2(float(sw(0) - 1.0)) + si : F2(3.f) * m.p * F2(float(sw(i))) + si;
        const F2 post = g[i] - (g[i] - geq) * ig + sg * G[i];
        sp_store2(gout, N, c, x, ys[sy(i) + 1], K.nx, (sy(i) > 0 && top) || (sy(i) < 0 && bot), i, post);
    }
}

// ---- Remarks 1 and 2 (M = 1, 2) ----
// g holds g_i - w_i a0 (a0 = 1 for Remark 1, p_0 for Remark 2: the rest state).
// d = rho - 1 (Remark 1) or p - p_0 (Remark 2); a = rho or p_0, the factor of
// s_i(u) in g^eq (Eq. 29bb, Eq. 29bd); both equilibria are d w_i + a s_i(u)
// after the shift. Sg and the force Fg are in the units of g (Remark 2: p_0 S_1,
// p_0 F_1).
template <int M, typename R>
__device__ __forceinline__ void sp1_moments(const SpConst& K, const R g[kQ], R S, R& d, R& a, R& ux, R& uy) {
    R m0 = g[0], jx = R(0), jy = R(0);
#pragma unroll
    for (int i = 1; i < kQ; ++i) {
        m0 += g[i];
        if (sx(i)) jx += sx(i) > 0 ? g[i] : -g[i];
        if (sy(i)) jy += sy(i) > 0 ? g[i] : -g[i];
    }
    if constexpr (M == 1) {
        d = m0 + R(0.5) * S;                       // Eq. 27aa
        a = R(1) + d;
        const R ir = sp_inv(a);
        ux = (jx + R(0.5) * R(K.fx)) * ir;         // Eq. 27a
        uy = (jy + R(0.5) * R(K.fy)) * ir;
    } else {
        d = m0 + R(K.hp0) * S;                     // p = sum g + p_0 S_1 / 2
        a = R(K.p0);
        ux = (jx + R(K.hp0fx)) * R(K.ip0);         // p_0 u = sum c g + p_0 F_1 / 2
        uy = (jy + R(K.hp0fy)) * R(K.ip0);
    }
}

// post-collision value of direction i (Eq. 24 with the force term of the remark)
template <int M, typename R>
__device__ __forceinline__ R sp1_post(const SpConst& K, int i, R gi, R d, R a, R ux, R uy, R S, R Qd) {
    const R sc = M == 1 ? R(1) : R(K.p0);          // S and F in the units of g
    const R fx = R(K.fx) * sc, fy = R(K.fy) * sc, Sg = S * sc;
    const R cu = R(sx(i)) * ux + R(sy(i)) * uy, cF = R(sx(i)) * fx + R(sy(i)) * fy;
    const R uF = ux * fx + uy * fy, uu = ux * ux + uy * uy;
    const R c2 = R(sx(i) * sx(i) + sy(i) * sy(i));
    const R si = R(sw(i)) * (R(3) * cu + R(4.5) * cu * cu - R(1.5) * uu);
    const R geq = d * R(sw(i)) + a * si;
    // (cc - c_s^2 I):(uF + Fu [- uu S] + Q div u I) / (2 c_s^4)
    //   = 9 (c.u)(c.F) - 3 u.F [- 4.5 ((c.u)^2 - u.u / 3) S] + 4.5 (|c|^2 - 2/3) Q div u
    R Gi = Sg + R(3) * cF + R(9) * cu * cF - R(3) * uF + R(4.5) * (c2 - R(2.0 / 3.0)) * Qd;
    if constexpr (M == 1) Gi = Gi - R(4.5) * (cu * cu - uu * R(1.0 / 3.0)) * Sg;   // the u u S of Remark 1
    return gi - (gi - geq) * R(K.inv_tau) + R(K.src) * (R(sw(i)) * Gi);
}

// The same for a direction i and its opposite j = opp(i): c_j = -c_i, so s_i and
// G_i split into a part even in c (shared) and an odd part (sign flipped).
template <int M, typename R>
__device__ __forceinline__ void sp1_post_pair(const SpConst& K, int i, R gi, R gj, R d, R a, R ux, R uy, R S,
                                              R Qd, R& pi, R& pj) {
    const R sc = M == 1 ? R(1) : R(K.p0);
    const R fx = R(K.fx) * sc, fy = R(K.fy) * sc, Sg = S * sc;
    const R cu = R(sx(i)) * ux + R(sy(i)) * uy, cF = R(sx(i)) * fx + R(sy(i)) * fy;
    const R uF = ux * fx + uy * fy, uu = ux * ux + uy * uy;
    const R c2 = R(sx(i) * sx(i) + sy(i) * sy(i));
    const R wi = R(sw(i));
    const R geq_e = d * wi + a * (wi * (R(4.5) * cu * cu - R(1.5) * uu)), geq_o = a * (wi * (R(3) * cu));
    R G_e = Sg + R(9) * cu * cF - R(3) * uF + R(4.5) * (c2 - R(2.0 / 3.0)) * Qd;
    if constexpr (M == 1) G_e = G_e - R(4.5) * (cu * cu - uu * R(1.0 / 3.0)) * Sg;   // the u u S of Remark 1
    G_e = wi * G_e;
    const R G_o = wi * (R(3) * cF);
    const R ig = R(K.inv_tau), sg = R(K.src);
    pi = gi - (gi - (geq_e + geq_o)) * ig + sg * (G_e + G_o);
    pj = gj - (gj - (geq_e - geq_o)) * ig + sg * (G_e - G_o);
}


template <int M, typename R>
__global__ void __launch_bounds__(256) sp1_moments_kernel(const R* __restrict__ gin, const R* __restrict__ src,
                                                          long long N, SpConst K, R* __restrict__ ufield) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    R g[kQ], d, a, ux, uy;
#pragma unroll
    for (int i = 0; i < kQ; ++i) g[i] = gin[i * N + c];
    sp1_moments<M>(K, g, src[c], d, a, ux, uy);
    ufield[c] = ux;
    ufield[N + c] = uy;
}

template <int M, typename R>
__global__ void __launch_bounds__(256) sp1_step_kernel(const R* __restrict__ gin, R* __restrict__ gout,
                                                       const R* __restrict__ src, const R* __restrict__ ufield,
                                                       long long N, SpConst K) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int x = (int)(c % K.nx), y = (int)(c / K.nx);
    R g[kQ], d, a, ux, uy;
#pragma unroll
    for (int i = 0; i < kQ; ++i) g[i] = gin[i * N + c];
    const R S = src[c];
    sp1_moments<M>(K, g, S, d, a, ux, uy);
    const int xs[3] = {x == 0 ? K.nx - 1 : x - 1, x, x == K.nx - 1 ? 0 : x + 1};
    // stencil rows: mirror at walls (reading Q7), wrap when periodic
    const int yst[3] = {y == 0 ? (K.walls ? 0 : K.ny - 1) : y - 1, y,
                        y == K.ny - 1 ? (K.walls ? K.ny - 1 : 0) : y + 1};
    R divu = R(0);   // Eq. 30a applied to u
#pragma unroll
    for (int i = 1; i < kQ; ++i) {
        const long long n = (long long)yst[sy(i) + 1] * K.nx + xs[sx(i) + 1];
        R cu = R(0);
        if (sx(i)) cu += sx(i) > 0 ? ufield[n] : -ufield[n];
        if (sy(i)) cu += sy(i) > 0 ? ufield[N + n] : -ufield[N + n];
        divu += R(sw(i)) * cu;
    }
    divu *= R(3);
    // Q = (2/d) a c_s^2 - xi / (tau_g - 1/2); K.Qd0 = -xi / (tau_g - 1/2)
    const R Qd = (a * R(1.0 / 3.0) + R(K.Qd0)) * divu;
    const bool bot = K.walls && y == 0, top = K.walls && y == K.ny - 1;
    const int ys[3] = {K.walls ? y - 1 : (y == 0 ? K.ny - 1 : y - 1), y,
                       K.walls ? y + 1 : (y == K.ny - 1 ? 0 : y + 1)};
    auto emit = [&](int i, R post) {
        long long dst;
        int k = i;
        if ((sy(i) > 0 && top) || (sy(i) < 0 && bot)) {
            dst = c;
            k = sopp(i);
        } else {
            dst = (long long)ys[sy(i) + 1] * K.nx + xs[sx(i) + 1];
        }
        gout[k * N + dst] = post;
    };
    emit(0, sp1_post<M>(K, 0, g[0], d, a, ux, uy, S, Qd));
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = pair2(q), j = sopp(i);
        R pi, pj;
        sp1_post_pair<M>(K, i, g[i], g[j], d, a, ux, uy, S, Qd, pi, pj);
        emit(i, pi);
        emit(j, pj);
    }
}

// FP32, two cells a thread (nx even)
template <int M>
__global__ void __launch_bounds__(256) sp1_moments_x2_kernel(const float* __restrict__ gin,
                                                             const float* __restrict__ src, int N, SpConst K,
                                                             float* __restrict__ ufield) {
    const int c = 2 * (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (c >= N) return;
    F2 g[kQ], d, a, ux, uy;
#pragma unroll
    for (int i = 0; i < kQ; ++i) g[i] = ld2(gin + i * N + c);
    sp1_moments<M>(K, g, ld2(src + c), d, a, ux, uy);
    st2(ufield + c, ux);
    st2(ufield + N + c, uy);
}

template <int M>
__global__ void __launch_bounds__(256, 3) sp1_step_x2_kernel(const float* __restrict__ gin, float* __restrict__ gout,
                                                          const float* __restrict__ src,
                                                          const float* __restrict__ ufield, int N, SpConst K) {
    const int c = 2 * (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (c >= N) return;
    const int x = (int)(c % K.nx), y = (int)(c / K.nx);
    F2 g[kQ], d, a, ux, uy;
#pragma unroll
    for (int i = 0; i < kQ; ++i) g[i] = ld2(gin + i * N + c);
    const F2 S = ld2(src + c);
    sp1_moments<M>(K, g, S, d, a, ux, uy);
    // stencil rows: mirror at walls (reading Q7), wrap when periodic
    const int yst[3] = {y == 0 ? (K.walls ? 0 : K.ny - 1) : y - 1, y,
                        y == K.ny - 1 ? (K.walls ? K.ny - 1 : 0) : y + 1};
    F2 divu(0.f);   // Eq. 30a applied to u
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const int row = yst[r] * K.nx;
        const Row2 UX(ufield + row, x, K.nx), UY(ufield + N + row, x, K.nx);
#pragma unroll
        for (int i = 1; i < kQ; ++i) {
            if (sy(i) + 1 != r) continue;
            F2 cu(0.f);
            if (sx(i)) cu += sx(i) > 0 ? UX.at(sx(i)) : -UX.at(sx(i));
            if (sy(i)) cu += sy(i) > 0 ? UY.at(sx(i)) : -UY.at(sx(i));
            divu += F2(float(sw(i))) * cu;
        }
    }
    divu *= F2(3.f);
    const F2 Qd = (a * F2(float(1.0 / 3.0)) + F2(float(K.Qd0))) * divu;
    const bool bot = K.walls && y == 0, top = K.walls && y == K.ny - 1;
    const int ys[3] = {K.walls ? y - 1 : (y == 0 ? K.ny - 1 : y - 1), y,
                       K.walls ? y + 1 : (y == K.ny - 1 ? 0 : y + 1)};
    auto emit = [&](int i, F2 post) {
        sp_store2(gout, N, c, x, ys[sy(i) + 1], K.nx, (sy(i) > 0 && top) || (sy(i) < 0 && bot), i, post);
    };
    emit(0, sp1_post<M>(K, 0, g[0], d, a, ux, uy, S, Qd));
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = pair2(q), j = sopp(i);
        F2 pi, pj;
        sp1_post_pair<M>(K, i, g[i], g[j], d, a, ux, uy, S, Qd, pi, pj);
        emit(i, pi);
        emit(j, pj);
    }
}

template <int M, typename R>
__global__ void sp1_fields_kernel(const R* __restrict__ g, const R* __restrict__ src, long long N, SpConst K,
                                  unsigned mask, double* __restrict__ out) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    R gc[kQ], d, a, ux, uy;
#pragma unroll
    for (int i = 0; i < kQ; ++i) gc[i] = g[i * N + c];
    sp1_moments<M>(K, gc, src[c], d, a, ux, uy);
    // Remark 1: p = rho c_s^2, rho = 1 + d; Remark 2: p = p_0 + d
    const double p = M == 1 ? (1.0 + double(d)) / 3.0 : K.p0 + double(d);
    int slot = 0;
    if (mask & LBM_FIELD_UX) out[(slot++) * N + c] = double(ux);
    if (mask & LBM_FIELD_UY) out[(slot++) * N + c] = double(uy);
    if (mask & LBM_FIELD_P) out[(slot++) * N + c] = p;
    if (M == 1 && (mask & LBM_FIELD_RHO)) out[(slot++) * N + c] = 1.0 + double(d);
}

// ---- Remark 4 scheme (on the Remark 3 model) ----
template <typename R>
__device__ __forceinline__ void sp4_u(const R f[kQ], R& ux, R& uy) {
    R jx = R(0), jy = R(0);
#pragma unroll
    for (int i = 1; i < kQ; ++i) {
        if (sx(i)) jx += sx(i) > 0 ? f[i] : -f[i];
        if (sy(i)) jy += sy(i) > 0 ? f[i] : -f[i];
    }
    ux = jx;
    uy = jy;
}

template <typename R>
__device__ __forceinline__ void sp4_force(const SpConst& K, R ux, R uy, R& Fx, R& Fy) {
    const R k = R(K.dl) + R(K.dq) * sp_sqrt(ux * ux + uy * uy);
    Fx = R(K.fx) - k * ux;
    Fy = R(K.fy) - k * uy;
}

// G_i of Remark 3 with force F at velocity u, direction i
template <typename R>
__device__ __forceinline__ R sp4_G(const SpConst& K, int i, R S, R ux, R uy, R Fx, R Fy) {
    const R cu = R(sx(i)) * ux + R(sy(i)) * uy, cF = R(sx(i)) * Fx + R(sy(i)) * Fy;
    const R c2 = R(sx(i) * sx(i) + sy(i) * sy(i));
    return R(sw(i)) * (S + R(3) * cF + R(9) * cu * cF - R(3) * (ux * Fx + uy * Fy) +
                       R(4.5) * (c2 - R(2.0 / 3.0)) * R(K.Qc) * S);
}

// sp4_G split into the part even in c and the odd part c.F / c_s^2 (times w_i)
template <typename R>
__device__ __forceinline__ void sp4_G_parts(const SpConst& K, int i, R S, R ux, R uy, R Fx, R Fy, R& e, R& o) {
    const R cu = R(sx(i)) * ux + R(sy(i)) * uy, cF = R(sx(i)) * Fx + R(sy(i)) * Fy;
    const R c2 = R(sx(i) * sx(i) + sy(i) * sy(i));
    e = R(sw(i)) * (S + R(9) * cu * cF - R(3) * (ux * Fx + uy * Fy) + R(4.5) * (c2 - R(2.0 / 3.0)) * R(K.Qc) * S);
    o = R(sw(i)) * (R(3) * cF);
}

// u = sum c f and F(u) of every cell, four planes (the update at x needs G at
// x + c_i, so these first; F is kept so that no neighbour evaluates the drag)
template <typename R>
__global__ void __launch_bounds__(256) sp4_moments_kernel(const R* __restrict__ fin, long long N,
                                                          SpConst K, R* __restrict__ unow) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    R f[kQ], ux, uy, Fx, Fy;
#pragma unroll
    for (int i = 0; i < kQ; ++i) f[i] = fin[i * N + c];
    sp4_u(f, ux, uy);
    sp4_force(K, ux, uy, Fx, Fy);
    unow[c] = ux;
    unow[N + c] = uy;
    unow[2 * N + c] = Fx;
    unow[3 * N + c] = Fy;
}

template <typename R>
__global__ void __launch_bounds__(256) sp4_step_kernel(const R* __restrict__ fin, R* __restrict__ fout,
                                                       const R* __restrict__ src, const R* __restrict__ unow,
                                                       const R* __restrict__ uprev, long long N, SpConst K) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int x = (int)(c % K.nx), y = (int)(c / K.nx);
    R f[kQ], ux, uy;
#pragma unroll
    for (int i = 0; i < kQ; ++i) f[i] = fin[i * N + c];
    const R S = src[c];
    sp4_u(f, ux, uy);
    const R Fx = unow[2 * N + c], Fy = unow[3 * N + c];
    R rest = R(0);
#pragma unroll
    for (int i = 1; i < kQ; ++i) rest += f[i];
    const R uu = ux * ux + uy * uy;
    const R G0 = sp4_G(K, 0, S, ux, uy, Fx, Fy);
    // Eq. 28 for the unshifted f: c_s^2 / (1 - w_0) = 3/5, s_0(u) = -(2/3) u.u, tau_g G_0
    const R p = R(0.6) * (rest - R(2.0 / 3.0) * uu + R(K.tau) * G0);
    const R upx = uprev[c], upy = uprev[N + c], Fpx = uprev[2 * N + c], Fpy = uprev[3 * N + c];
    const R ig = R(K.inv_tau);
    const bool bot = K.walls && y == 0, top = K.walls && y == K.ny - 1;
    const int xs[3] = {x == 0 ? K.nx - 1 : x - 1, x, x == K.nx - 1 ? 0 : x + 1};
    const int ys[3] = {K.walls ? y - 1 : (y == 0 ? K.ny - 1 : y - 1), y,
                       K.walls ? y + 1 : (y == K.ny - 1 ? 0 : y + 1)};
    // G_i(x + c_i, t): the destination cell, mirrored about a wall
    auto Gnb = [&](int i) {
        const bool wall = (sy(i) > 0 && top) || (sy(i) < 0 && bot);
        const long long n = (long long)(wall ? y : ys[sy(i) + 1]) * K.nx + xs[sx(i) + 1];
        return sp4_G(K, i, src[n], unow[n], unow[N + n], unow[2 * N + n], unow[3 * N + n]);
    };
    // to x + c_i, or (wall) back into this cell as opp(i) after the bounce-back of g = f - G/2
    auto emit = [&](int i, R post, R Gn, R Gopp) {
        if ((sy(i) > 0 && top) || (sy(i) < 0 && bot))
            fout[sopp(i) * N + c] = post - R(0.5) * Gn + R(0.5) * Gopp;
        else
            fout[i * N + (long long)ys[sy(i) + 1] * K.nx + xs[sx(i) + 1]] = post;
    };
    {   // rest direction: its destination is this cell
        const R geq = R(3) * p * (R(sw(0)) - R(1)) + R(sw(0)) * (-R(1.5) * uu);
        const R Gp = sp4_G(K, 0, S, upx, upy, Fpx, Fpy);
        emit(0, f[0] - (f[0] - geq) * ig + G0 + R(0.5) * (G0 - Gp), G0, G0);
    }
    // opposite pairs: G at t and t - 1 and s_i split into parts even and odd in c
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = pair2(q), j = sopp(i);
        const R wi = R(sw(i));
        const R cu = R(sx(i)) * ux + R(sy(i)) * uy;
        const R ge = R(3) * p * wi + wi * (R(4.5) * cu * cu - R(1.5) * uu), go = wi * (R(3) * cu);
        R Ge, Go, Gpe, Gpo;
        sp4_G_parts(K, i, S, ux, uy, Fx, Fy, Ge, Go);
        sp4_G_parts(K, i, S, upx, upy, Fpx, Fpy, Gpe, Gpo);
        const R Gi = Ge + Go, Gj = Ge - Go, Gni = Gnb(i), Gnj = Gnb(j);
        emit(i, f[i] - (f[i] - (ge + go)) * ig + Gi + R(0.5) * (Gni - (Gpe + Gpo)), Gni, Gj);
        emit(j, f[j] - (f[j] - (ge - go)) * ig + Gj + R(0.5) * (Gnj - (Gpe - Gpo)), Gnj, Gi);
    }
}

// Remark 4 scheme, FP32, two cells a thread (nx even)
__global__ void __launch_bounds__(256) sp4_moments_x2_kernel(const float* __restrict__ fin, int N,
                                                             SpConst K, float* __restrict__ unow) {
    const int c = 2 * (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (c >= N) return;
    F2 f[kQ], ux, uy, Fx, Fy;
#pragma unroll
    for (int i = 0; i < kQ; ++i) f[i] = ld2(fin + i * N + c);
    sp4_u(f, ux, uy);
    sp4_force(K, ux, uy, Fx, Fy);
    st2(unow + c, ux);
    st2(unow + N + c, uy);
    st2(unow + 2 * N + c, Fx);
    st2(unow + 3 * N + c, Fy);
}

__global__ void __launch_bounds__(256) sp4_step_x2_kernel(const float* __restrict__ fin, float* __restrict__ fout,
                                                          const float* __restrict__ src,
                                                          const float* __restrict__ unow,
                                                          const float* __restrict__ uprev, int N, SpConst K) {
    const int c = 2 * (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (c >= N) return;
    const int x = (int)(c % K.nx), y = (int)(c / K.nx);
    F2 f[kQ], ux, uy;
#pragma unroll
    for (int i = 0; i < kQ; ++i) f[i] = ld2(fin + i * N + c);
    const F2 S = ld2(src + c);
    sp4_u(f, ux, uy);
    const F2 Fx = ld2(unow + 2 * N + c), Fy = ld2(unow + 3 * N + c);
    F2 rest(0.f);
#pragma unroll
    for (int i = 1; i < kQ; ++i) rest += f[i];
    const F2 uu = ux * ux + uy * uy;
    const F2 G0 = sp4_G(K, 0, S, ux, uy, Fx, Fy);
    const F2 p = F2(0.6f) * (rest - F2(float(2.0 / 3.0)) * uu + F2(float(K.tau)) * G0);
    const F2 upx = ld2(uprev + c), upy = ld2(uprev + N + c), Fpx = ld2(uprev + 2 * N + c),
             Fpy = ld2(uprev + 3 * N + c);
    const F2 ig(float(K.inv_tau));
    const bool bot = K.walls && y == 0, top = K.walls && y == K.ny - 1;
    const int ys[3] = {K.walls ? y - 1 : (y == 0 ? K.ny - 1 : y - 1), y,
                       K.walls ? y + 1 : (y == K.ny - 1 ? 0 : y + 1)};
    // rows of the destinations x + c_i for G_i(x + c_i, t): mirrored about a wall
    const int yst[3] = {y == 0 ? (K.walls ? 0 : K.ny - 1) : y - 1, y,
                        y == K.ny - 1 ? (K.walls ? K.ny - 1 : 0) : y + 1};
    const int xl[3] = {x == 0 ? K.nx - 1 : x - 1, x, x + 1};   // left lane's x + c_x
    const int xr[3] = {x, x + 1, x + 2 == K.nx ? 0 : x + 2};   // right lane's
    // G_i(x + c_i, t) from the destination's u, F and S
    auto Gnb = [&](int i) {
        const int row = yst[sy(i) + 1] * K.nx;
        const int a = row + xl[sx(i) + 1], b = row + xr[sx(i) + 1];
        auto nb = [&](const float* pl) { return sx(i) == 0 ? ld2(pl + a) : F2(pl[a], pl[b]); };
        return sp4_G(K, i, nb(src), nb(unow), nb(unow + N), nb(unow + 2 * N), nb(unow + 3 * N));
    };
    {   // rest direction: never crosses a wall; its destination is this cell
        const F2 Gp = sp4_G(K, 0, S, upx, upy, Fpx, Fpy);
        const F2 geq = F2(3.f) * p * F2(float(sw(0) - 1.0)) + float(sw(0)) * (-F2(1.5f) * uu);
        sp_store2(fout, N, c, x, y, K.nx, false, 0, f[0] - (f[0] - geq) * ig + G0 + F2(0.5f) * (G0 - Gp));
    }
    // opposite pairs (i, j = opp(i)): G of this cell at t and t - 1 and s_i split
    // into parts even and odd in c
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = pair2(q), j = sopp(i);
        const float wi = float(sw(i));
        const F2 cu = float(sx(i)) * ux + float(sy(i)) * uy;
        const F2 ge = F2(3.f * wi) * p + wi * (F2(4.5f) * cu * cu - F2(1.5f) * uu), go = wi * (F2(3.f) * cu);
        F2 Ge, Go, Gpe, Gpo;
        sp4_G_parts(K, i, S, ux, uy, Fx, Fy, Ge, Go);
        sp4_G_parts(K, i, S, upx, upy, Fpx, Fpy, Gpe, Gpo);
        const F2 Gi = Ge + Go, Gj = Ge - Go;
        const F2 Gni = Gnb(i), Gnj = Gnb(j);
        F2 pi = f[i] - (f[i] - (ge + go)) * ig + Gi + F2(0.5f) * (Gni - (Gpe + Gpo));
        F2 pj = f[j] - (f[j] - (ge - go)) * ig + Gj + F2(0.5f) * (Gnj - (Gpe - Gpo));
        // bounce-back of g = f - G/2: leaves as i with G_i(x + c_i), returns as opp(i)
        const bool bi = (sy(i) > 0 && top) || (sy(i) < 0 && bot), bj = (sy(j) > 0 && top) || (sy(j) < 0 && bot);
        if (bi) pi = pi - F2(0.5f) * Gni + F2(0.5f) * Gj;
        if (bj) pj = pj - F2(0.5f) * Gnj + F2(0.5f) * Gi;
        sp_store2(fout, N, c, x, ys[sy(i) + 1], K.nx, bi, i, pi);
        sp_store2(fout, N, c, x, ys[sy(j) + 1], K.nx, bj, j, pj);
    }
}

template <typename R>
__global__ void sp4_fields_kernel(const R* __restrict__ f, const R* __restrict__ src, long long N, SpConst K,
                                  unsigned mask, double* __restrict__ out) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    R fc[kQ], ux, uy, Fx, Fy;
#pragma unroll
    for (int i = 0; i < kQ; ++i) fc[i] = f[i * N + c];
    sp4_u(fc, ux, uy);
    sp4_force(K, ux, uy, Fx, Fy);
    R rest = R(0);
#pragma unroll
    for (int i = 1; i < kQ; ++i) rest += fc[i];
    const R G0 = sp4_G(K, 0, src[c], ux, uy, Fx, Fy);
    const R p = R(0.6) * (rest - R(2.0 / 3.0) * (ux * ux + uy * uy) + R(K.tau) * G0);
    int slot = 0;
    if (mask & LBM_FIELD_UX) out[(slot++) * N + c] = double(ux);
    if (mask & LBM_FIELD_UY) out[(slot++) * N + c] = double(uy);
    if (mask & LBM_FIELD_P) out[(slot++) * N + c] = double(p);
}

// populations g_i = stored + w_i, widened to FP64
template <typename R>
__global__ void sp1_widen_kernel(const R* __restrict__ in, double* __restrict__ out, long long N, double a0) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
#pragma unroll
    for (int i = 0; i < kQ; ++i) out[i * N + c] = double(in[i * N + c]) + sw(i) * a0;
}

template <typename R>
__global__ void sp_fields_kernel(const R* __restrict__ g, const R* __restrict__ src, long long N, SpConst K,
                                 unsigned mask, double* __restrict__ out) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    R gc[kQ], G[kQ];
#pragma unroll
    for (int i = 0; i < kQ; ++i) gc[i] = g[i * N + c];
    const SpCell<R> m = sp_moments(K, gc, src[c], G);
    int slot = 0;
    if (mask & LBM_FIELD_UX) out[(slot++) * N + c] = double(m.ux);
    if (mask & LBM_FIELD_UY) out[(slot++) * N + c] = double(m.uy);
    if (mask & LBM_FIELD_P) out[(slot++) * N + c] = double(m.p);
}

template <typename R>
__global__ void sp_convert_kernel(const double* __restrict__ in, R* __restrict__ out, long long n) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) out[c] = R(in[c]);
}

template <typename R>
__global__ void sp_fill_kernel(R* __restrict__ out, double v, long long n) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) out[c] = R(v);
}

template <typename R>
__global__ void sp_widen_kernel(const R* __restrict__ in, double* __restrict__ out, long long n) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) out[c] = double(in[c]);
}

}  // namespace

struct lbm_sp_ctx {
    lbm_sp_params p;
    int form = 0;                      // LBM_F64 or LBM_F32
    long long N = 0;
    void* g[2] = {nullptr, nullptr};
    void* src = nullptr;
    void* ufield = nullptr;            // Remark 1: u of the current step (2 planes);
                                       // Remark 4 scheme: u, F(u) at t and t - 1 (2 x 4 planes)
    int uprev = 0;                     // Remark 4 scheme: which half of ufield holds u at t - 1
    double* d_tmp = nullptr;           // staging for inputs and outputs
    int cur = 0;
    bool ready = false;
    long long time = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    SpConst K{};
    std::string err;
};

namespace {

lbm_status sp_fail(lbm_sp_ctx* c, lbm_status st, const std::string& m) {
    if (c) c->err = m;
    return st;
}
lbm_status sp_cuda(lbm_sp_ctx* c, cudaError_t e, const char* what) {
    return sp_fail(c, LBM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
size_t sp_elem(int form) { return form == LBM_F64 ? 8 : 4; }
int blocks(long long n) { return (int)((n + 255) / 256); }

void sp_release(lbm_sp_ctx* c) {
    cudaFree(c->g[0]);
    cudaFree(c->g[1]);
    cudaFree(c->src);
    cudaFree(c->ufield);
    cudaFree(c->d_tmp);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
}

// Remarks 1 and 2: u, then the collision
template <int M>
void sp1_enqueue(lbm_sp_ctx* c) {
    if (c->form == LBM_F64) {
        const double* gi = static_cast<const double*>(c->g[c->cur]);
        double* uf = static_cast<double*>(c->ufield);
        sp1_moments_kernel<M, double><<<blocks(c->N), 256, 0, c->stream>>>(
            gi, static_cast<const double*>(c->src), c->N, c->K, uf);
        sp1_step_kernel<M, double><<<blocks(c->N), 256, 0, c->stream>>>(
            gi, static_cast<double*>(c->g[1 - c->cur]), static_cast<const double*>(c->src), uf, c->N, c->K);
        return;
    }
    const float* gi = static_cast<const float*>(c->g[c->cur]);
    float* uf = static_cast<float*>(c->ufield);
    if (c->p.nx % 2 == 0) {   // two cells a thread
        sp1_moments_x2_kernel<M><<<blocks(c->N / 2), 256, 0, c->stream>>>(
            gi, static_cast<const float*>(c->src), c->N, c->K, uf);
        sp1_step_x2_kernel<M><<<blocks(c->N / 2), 256, 0, c->stream>>>(
            gi, static_cast<float*>(c->g[1 - c->cur]), static_cast<const float*>(c->src), uf, c->N, c->K);
    } else {
        sp1_moments_kernel<M, float><<<blocks(c->N), 256, 0, c->stream>>>(
            gi, static_cast<const float*>(c->src), c->N, c->K, uf);
        sp1_step_kernel<M, float><<<blocks(c->N), 256, 0, c->stream>>>(
            gi, static_cast<float*>(c->g[1 - c->cur]), static_cast<const float*>(c->src), uf, c->N, c->K);
    }
}

template <int M>
void sp1_fields(lbm_sp_ctx* c, unsigned mask) {
    if (c->form == LBM_F64)
        sp1_fields_kernel<M, double><<<blocks(c->N), 256, 0, c->stream>>>(
            static_cast<const double*>(c->g[c->cur]), static_cast<const double*>(c->src), c->N, c->K, mask, c->d_tmp);
    else
        sp1_fields_kernel<M, float><<<blocks(c->N), 256, 0, c->stream>>>(
            static_cast<const float*>(c->g[c->cur]), static_cast<const float*>(c->src), c->N, c->K, mask, c->d_tmp);
}

}  // namespace

extern "C" {

lbm_status lbm_sp_create(const lbm_sp_params* params, int precision, void* cuda_stream, lbm_sp_ctx** out) {
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    if (!params) return LBM_EINVAL;
    const lbm_sp_params& p = *params;
    if (p.nx < 3 || p.ny < 3 || (long long)p.nx * p.ny >= (1LL << 31) / 9) return LBM_EINVAL;
    if (p.bc_y != LBM_BC_PERIODIC && p.bc_y != LBM_BC_BOUNCEBACK) return LBM_EINVAL;
    if (p.model != LBM_SP_INCOMPRESSIBLE_SOURCE && p.model != LBM_SP_NEARLY_INCOMPRESSIBLE &&
        p.model != LBM_SP_HE_INCOMPRESSIBLE)
        return LBM_EINVAL;
    if (p.model == LBM_SP_HE_INCOMPRESSIBLE && !(std::isfinite(p.p0) && p.p0 > 0)) return LBM_EINVAL;
    if ((p.scheme != LBM_SP_SCHEME_EQ24 && p.scheme != LBM_SP_SCHEME_REMARK4) || p.reserved != 0) return LBM_EINVAL;
    if (!(std::isfinite(p.drag_lin) && p.drag_lin >= 0) || !(std::isfinite(p.drag_quad) && p.drag_quad >= 0))
        return LBM_EINVAL;
    // a velocity-dependent force makes Eq. 27a implicit: it needs the Remark 4 scheme,
    // which is built on the Remark 3 model
    if (p.scheme == LBM_SP_SCHEME_EQ24 && (p.drag_lin != 0 || p.drag_quad != 0)) return LBM_EINVAL;
    if (p.scheme == LBM_SP_SCHEME_REMARK4 && p.model != LBM_SP_INCOMPRESSIBLE_SOURCE) return LBM_EINVAL;
    if (!(std::isfinite(p.nu) && p.nu > 0) || !(std::isfinite(p.xi) && p.xi >= 0) || !std::isfinite(p.force_x) ||
        !std::isfinite(p.force_y))
        return LBM_EINVAL;
    if (precision != LBM_F64 && precision != LBM_F32) return LBM_EINVAL;
    lbm_sp_ctx* c = new lbm_sp_ctx();
    c->p = p;
    c->form = precision;
    c->N = (long long)p.nx * p.ny;
    const double tau = 3.0 * p.nu + 0.5;
    c->K = SpConst{p.nx, p.ny, p.bc_y == LBM_BC_BOUNCEBACK ? 1 : 0, 1.0 / tau, 1.0 - 0.5 / tau, tau - 0.5,
                   1.0 / 3.0 - p.xi / (tau - 0.5), p.force_x, p.force_y, p.drag_lin, p.drag_quad, p.p0,
                   tau, -p.xi / (tau - 0.5), 0.5 * p.p0, p.p0 > 0 ? 1.0 / p.p0 : 0.0, 0.5 * p.p0 * p.force_x,
                   0.5 * p.p0 * p.force_y};
    const size_t e = sp_elem(precision);
    cudaError_t r;
    if ((r = cudaMalloc(&c->g[0], kQ * c->N * e)) != cudaSuccess ||
        (r = cudaMalloc(&c->g[1], kQ * c->N * e)) != cudaSuccess ||
        (r = cudaMalloc(&c->src, c->N * e)) != cudaSuccess ||
        ((p.model == LBM_SP_NEARLY_INCOMPRESSIBLE || p.model == LBM_SP_HE_INCOMPRESSIBLE) &&
         (r = cudaMalloc(&c->ufield, 2 * c->N * e)) != cudaSuccess) ||
        (p.scheme == LBM_SP_SCHEME_REMARK4 && (r = cudaMalloc(&c->ufield, 8 * c->N * e)) != cudaSuccess) ||
        (r = cudaMalloc((void**)&c->d_tmp, kQ * c->N * sizeof(double))) != cudaSuccess) {
        sp_release(c);
        delete c;
        return r == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
    }
    if (cuda_stream) {
        c->stream = static_cast<cudaStream_t>(cuda_stream);
    } else if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) == cudaSuccess) {
        c->own_stream = true;
    } else {
        sp_release(c);
        delete c;
        return LBM_ECUDA;
    }
    *out = c;
    return LBM_OK;
}

lbm_status lbm_sp_init(lbm_sp_ctx* c, const double* source_host) {
    if (!c) return LBM_EINVAL;
    if (!source_host) return sp_fail(c, LBM_EINVAL, "source is NULL");
    cudaError_t r;
    if ((r = cudaMemcpyAsync(c->d_tmp, source_host, c->N * sizeof(double), cudaMemcpyHostToDevice,
                             c->stream)) != cudaSuccess)
        return sp_cuda(c, r, "source upload");
    if (c->form == LBM_F64) {
        sp_convert_kernel<double><<<blocks(c->N), 256, 0, c->stream>>>(c->d_tmp, static_cast<double*>(c->src), c->N);
    } else {
        sp_convert_kernel<float><<<blocks(c->N), 256, 0, c->stream>>>(c->d_tmp, static_cast<float*>(c->src), c->N);
    }
    c->cur = 0;
    // at rest: Remark 3 g^eq = rho_0 delta_i0 (g_0 stored shifted by rho_0);
    // Remark 1 g^eq = w_i at rho = 1, Remark 2 w_i p_0 (stored shifted by
    // them) -- zero in every case
    if ((r = cudaMemsetAsync(c->g[0], 0, kQ * c->N * sp_elem(c->form), c->stream)) != cudaSuccess)
        return sp_cuda(c, r, "state reset");
    // Remark 4 scheme: u at t = -1 is u at t = 0 = 0
    c->uprev = 0;
    if (c->p.scheme == LBM_SP_SCHEME_REMARK4 &&
        (r = cudaMemsetAsync(c->ufield, 0, 8 * c->N * sp_elem(c->form), c->stream)) != cudaSuccess)
        return sp_cuda(c, r, "state reset");
    if (c->p.scheme == LBM_SP_SCHEME_REMARK4) {   // F(u = 0) = F_0 at t = -1
        const double F0[2] = {c->p.force_x, c->p.force_y};
        for (int a = 0; a < 2; ++a) {
            if (c->form == LBM_F64)
                sp_fill_kernel<double><<<blocks(c->N), 256, 0, c->stream>>>(
                    static_cast<double*>(c->ufield) + (2 + a) * c->N, F0[a], c->N);
            else
                sp_fill_kernel<float><<<blocks(c->N), 256, 0, c->stream>>>(
                    static_cast<float*>(c->ufield) + (2 + a) * c->N, F0[a], c->N);
        }
    }
    if ((r = cudaStreamSynchronize(c->stream)) != cudaSuccess) return sp_cuda(c, r, "init");
    if ((r = cudaGetLastError()) != cudaSuccess) return sp_cuda(c, r, "init kernel");
    c->ready = true;
    c->time = 0;
    return LBM_OK;
}

lbm_status lbm_sp_step(lbm_sp_ctx* c, int nsteps) {
    if (!c) return LBM_EINVAL;
    if (nsteps < 0) return sp_fail(c, LBM_EINVAL, "nsteps < 0");
    if (!c->ready) return sp_fail(c, LBM_ESTATE, "not initialised");
    const bool m1 = c->p.model == LBM_SP_NEARLY_INCOMPRESSIBLE, m2 = c->p.model == LBM_SP_HE_INCOMPRESSIBLE;
    const bool r4 = c->p.scheme == LBM_SP_SCHEME_REMARK4;
    for (int s = 0; s < nsteps; ++s) {
        if (r4) {
            const long long h = 4 * c->N;
            const int un = 1 - c->uprev;
            if (c->form == LBM_F64) {
                const double* fi = static_cast<const double*>(c->g[c->cur]);
                double* u = static_cast<double*>(c->ufield);
                sp4_moments_kernel<double><<<blocks(c->N), 256, 0, c->stream>>>(fi, c->N, c->K, u + un * h);
                sp4_step_kernel<double><<<blocks(c->N), 256, 0, c->stream>>>(
                    fi, static_cast<double*>(c->g[1 - c->cur]), static_cast<const double*>(c->src), u + un * h,
                    u + c->uprev * h, c->N, c->K);
            } else {
                const float* fi = static_cast<const float*>(c->g[c->cur]);
                float* u = static_cast<float*>(c->ufield);
                if (c->p.nx % 2 == 0) {   // two cells a thread
                    sp4_moments_x2_kernel<<<blocks(c->N / 2), 256, 0, c->stream>>>(fi, c->N, c->K, u + un * h);
                    sp4_step_x2_kernel<<<blocks(c->N / 2), 256, 0, c->stream>>>(
                        fi, static_cast<float*>(c->g[1 - c->cur]), static_cast<const float*>(c->src), u + un * h,
                        u + c->uprev * h, c->N, c->K);
                } else {
                    sp4_moments_kernel<float><<<blocks(c->N), 256, 0, c->stream>>>(fi, c->N, c->K, u + un * h);
                    sp4_step_kernel<float><<<blocks(c->N), 256, 0, c->stream>>>(
                        fi, static_cast<float*>(c->g[1 - c->cur]), static_cast<const float*>(c->src), u + un * h,
                        u + c->uprev * h, c->N, c->K);
                }
            }
            c->uprev = un;
        } else if (m1) {
            sp1_enqueue<1>(c);
        } else if (m2) {
            sp1_enqueue<2>(c);        } else if (c->form == LBM_F64)
            sp_step_kernel<double><<<blocks(c->N), 256, 0, c->stream>>>(
                static_cast<const double*>(c->g[c->cur]), static_cast<double*>(c->g[1 - c->cur]),
                static_cast<const double*>(c->src), c->N, c->K);
        else if (c->p.nx % 2 == 0)   // two cells a thread
            sp_step_x2_kernel<<<blocks(c->N / 2), 256, 0, c->stream>>>(
                static_cast<const float*>(c->g[c->cur]), static_cast<float*>(c->g[1 - c->cur]),
                static_cast<const float*>(c->src), c->N, c->K);
        else
            sp_step_kernel<float><<<blocks(c->N), 256, 0, c->stream>>>(
                static_cast<const float*>(c->g[c->cur]), static_cast<float*>(c->g[1 - c->cur]),
                static_cast<const float*>(c->src), c->N, c->K);
        c->cur ^= 1;
    }
    c->time += nsteps;
    const cudaError_t r = cudaGetLastError();
    return r == cudaSuccess ? LBM_OK : sp_cuda(c, r, "step kernel");
}

lbm_status lbm_sp_get_fields(lbm_sp_ctx* c, unsigned mask, double* host_out) {
    if (!c) return LBM_EINVAL;
    const bool m1 = c->p.model == LBM_SP_NEARLY_INCOMPRESSIBLE, m2 = c->p.model == LBM_SP_HE_INCOMPRESSIBLE;
    const unsigned ok = LBM_FIELD_UX | LBM_FIELD_UY | LBM_FIELD_P | (m1 ? LBM_FIELD_RHO : 0u);
    if (!host_out || mask == 0 || (mask & ~ok)) return sp_fail(c, LBM_EINVAL, "bad mask or output");
    if (!c->ready) return sp_fail(c, LBM_ESTATE, "not initialised");
    const int nf = ((mask & LBM_FIELD_UX) ? 1 : 0) + ((mask & LBM_FIELD_UY) ? 1 : 0) + ((mask & LBM_FIELD_P) ? 1 : 0) +
                   ((mask & LBM_FIELD_RHO) ? 1 : 0);
    if (c->p.scheme == LBM_SP_SCHEME_REMARK4 && c->form == LBM_F64)
        sp4_fields_kernel<double><<<blocks(c->N), 256, 0, c->stream>>>(
            static_cast<const double*>(c->g[c->cur]), static_cast<const double*>(c->src), c->N, c->K, mask, c->d_tmp);
    else if (c->p.scheme == LBM_SP_SCHEME_REMARK4)
        sp4_fields_kernel<float><<<blocks(c->N), 256, 0, c->stream>>>(
            static_cast<const float*>(c->g[c->cur]), static_cast<const float*>(c->src), c->N, c->K, mask, c->d_tmp);
    else if (m1)
        sp1_fields<1>(c, mask);
    else if (m2)
        sp1_fields<2>(c, mask);
    else if (c->form == LBM_F64)
        sp_fields_kernel<double><<<blocks(c->N), 256, 0, c->stream>>>(
            static_cast<const double*>(c->g[c->cur]), static_cast<const double*>(c->src), c->N, c->K, mask, c->d_tmp);
    else
        sp_fields_kernel<float><<<blocks(c->N), 256, 0, c->stream>>>(
            static_cast<const float*>(c->g[c->cur]), static_cast<const float*>(c->src), c->N, c->K, mask, c->d_tmp);
    cudaError_t r;
    if ((r = cudaMemcpyAsync(host_out, c->d_tmp, nf * c->N * sizeof(double), cudaMemcpyDeviceToHost,
                             c->stream)) != cudaSuccess)
        return sp_cuda(c, r, "fields read-back");
    if ((r = cudaStreamSynchronize(c->stream)) != cudaSuccess) return sp_cuda(c, r, "fields");
    return LBM_OK;
}

lbm_status lbm_sp_get_populations(lbm_sp_ctx* c, double* host_g) {
    if (!c) return LBM_EINVAL;
    if (!host_g) return sp_fail(c, LBM_EINVAL, "output is NULL");
    if (!c->ready) return sp_fail(c, LBM_ESTATE, "not initialised");
    const long long n = kQ * c->N;
    const bool shifted = c->p.model == LBM_SP_NEARLY_INCOMPRESSIBLE || c->p.model == LBM_SP_HE_INCOMPRESSIBLE;
    const double a0 = c->p.model == LBM_SP_HE_INCOMPRESSIBLE ? c->p.p0 : 1.0;   // the stored shift w_i a0
    if (shifted && c->form == LBM_F64)
        sp1_widen_kernel<double><<<blocks(c->N), 256, 0, c->stream>>>(static_cast<const double*>(c->g[c->cur]),
                                                                      c->d_tmp, c->N, a0);
    else if (shifted)
        sp1_widen_kernel<float><<<blocks(c->N), 256, 0, c->stream>>>(static_cast<const float*>(c->g[c->cur]),
                                                                     c->d_tmp, c->N, a0);
    else if (c->form == LBM_F64)
        sp_widen_kernel<double><<<blocks(n), 256, 0, c->stream>>>(static_cast<const double*>(c->g[c->cur]), c->d_tmp, n);
    else
        sp_widen_kernel<float><<<blocks(n), 256, 0, c->stream>>>(static_cast<const float*>(c->g[c->cur]), c->d_tmp, n);
    cudaError_t r;
    if ((r = cudaMemcpyAsync(host_g, c->d_tmp, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess)
        return sp_cuda(c, r, "populations read-back");
    if ((r = cudaStreamSynchronize(c->stream)) != cudaSuccess) return sp_cuda(c, r, "populations");
    return LBM_OK;
}

const char* lbm_sp_last_error(const lbm_sp_ctx* c) { return c ? c->err.c_str() : "null context"; }

void lbm_sp_destroy(lbm_sp_ctx* c) {
    if (!c) return;
    sp_release(c);
    delete c;
}

}  // extern "C"
