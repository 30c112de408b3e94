// lbm_aux.cuh -- the kernels around the time step: the initial state, the
// macroscopic fields for read-back, the FP64 diagnostics and the population
// dump. Off the hot loop; they reuse the cell arithmetic of lbm_device.cuh.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

// ---------------------------------------------------------------------------
// Initial state (reading Q6): h = h^eq(phi0, mu0, u = 0), g = g^eq(p = 0, u = 0)
// (all zero with rho_0 = 0), phi*u of the previous step 0, p 0.
template <int FORM>
__global__ void init_kernel(const StepArgs a, const double* __restrict__ phi0, int instance) {
    using F = Form<FORM>;
    using R = typename F::R;
    using AT = typename F::AT;
    Consts<R> C;
    C.load(a.inst[instance]);
    PopIO<F> io;
    io.hout = static_cast<typename F::HT*>(a.h_out);
    io.h0out = static_cast<float2*>(a.h0_out);
    io.gout = static_cast<typename F::GT*>(a.g_out);
    io.S = a.S; io.hs = C.hs; io.ihs = C.ihs; io.gs = C.gs; io.igs = C.igs;
    AT* phiu = static_cast<AT*>(a.phiu);
    AT* p0 = static_cast<AT*>(a.p_out);
    AT* p1 = static_cast<AT*>(const_cast<void*>(a.p_in));
    const int n = C.nx * C.ny;
    for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < n; cell += gridDim.x * blockDim.x) {
        const int x = cell % C.nx, y = cell / C.nx;
        Nbr<R> nb;
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int yy = y + dy, xx = x + dx;
                xx = xx < 0 ? xx + C.nx : (xx >= C.nx ? xx - C.nx : xx);
                if (C.walls) yy = yy < 0 ? -1 - yy : (yy >= C.ny ? 2 * C.ny - 1 - yy : yy);
                else yy = yy < 0 ? yy + C.ny : (yy >= C.ny ? yy - C.ny : yy);
                nb.z[dy + 1][dx + 1] = R(phi0[yy * C.nx + xx]);
            }
        const R phi = nb.z[1][1];
        const R mu = chem_pot(C, phi, nb.lap());
        const R etamu = C.eta * mu;
        const long long c = C.base + cell;
        R hv[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) hv[i] = (i == 0) ? phi + (w_of<R>(0) - R(1)) * etamu : w_of<R>(i) * etamu;
        if constexpr (F::cons) {
            // h_0 = phi_0 - sum of the stored h_1..8, exactly as a float pair
            double rest = 0.0;
#pragma unroll
            for (int i = 1; i < 9; ++i) { hv[i] = io.round_h(hv[i]); rest += double(hv[i]); }
            const double h0 = phi0[cell] - rest;
            const float hi = float(h0);
            io.store_h0(c, make_float2(hi, float(h0 - double(hi))));
        } else {
            io.store_h(0, c, hv[0]);
        }
#pragma unroll
        for (int i = 1; i < 9; ++i) io.store_h(i, c, hv[i]);
#pragma unroll
        for (int i = 0; i < 9; ++i) io.store_g(i, c, R(0));
        phiu[c] = AT(0);
        phiu[a.S + c] = AT(0);
        p0[c] = AT(0);
        p1[c] = AT(0);
    }
}

// ---------------------------------------------------------------------------
// Macroscopic fields and diagnostics of one instance, in three passes over
// global memory (phi, then mu, then everything else) -- off the hot loop. They
// compute in FP64 whatever the storage form: the stored populations convert to
// FP64 exactly (phi of the conservative forms from its two-float h_0 to about
// 2^-48), so the fields, sums and the Laplace pressure P of Sec. 4.2 measure the
// stored state without adding FP32 rounding of their own.
template <int FORM>
__global__ void phi_pass(const AuxArgs a) {
    using F = Form<FORM>;
    using R = typename F::R;
    Consts<R> C;
    C.load(a.inst[a.instance]);
    PopIO<F> io;
    io.hin = static_cast<const typename F::HT*>(a.h);
    io.h0in = static_cast<const float2*>(a.h0);
    io.S = a.S; io.hs = C.hs; io.ihs = C.ihs;
    const int n = C.nx * C.ny;
    for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < n; cell += gridDim.x * blockDim.x) {
        const long long c = C.base + cell;
        R hv[9], lo;
        const R phi = io.phi_of(c, hv, lo);
        a.tmp_phi[cell] = double(phi) + double(lo);
    }
}

template <typename R>
__device__ __forceinline__ void gather(const double* f, int nx, int ny, int walls, int x, int y,
                                       Nbr<R>& nb) {
    for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
            int yy = y + dy, xx = x + dx;
            xx = xx < 0 ? xx + nx : (xx >= nx ? xx - nx : xx);
            if (walls) yy = yy < 0 ? -1 - yy : (yy >= ny ? 2 * ny - 1 - yy : yy);
            else yy = yy < 0 ? yy + ny : (yy >= ny ? yy - ny : yy);
            nb.z[dy + 1][dx + 1] = R(f[yy * nx + xx]);
        }
}

template <int FORM>
__global__ void mu_pass(const AuxArgs a) {
    using R = double;
    Consts<R> C;
    C.load(a.inst[a.instance]);
    const int n = C.nx * C.ny;
    for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < n; cell += gridDim.x * blockDim.x) {
        Nbr<R> nb;
        gather(a.tmp_phi, C.nx, C.ny, C.walls, cell % C.nx, cell / C.nx, nb);
        a.tmp_mu[cell] = double(chem_pot(C, nb.z[1][1], nb.lap()));
    }
}

// Everything one cell's macroscopic stage produces, plus the Laplace-law P of Sec. 4.2.
template <int FORM>
__device__ __forceinline__ void cell_fields(const AuxArgs& a, const Consts<double>& C, int cell, double out[7],
                                            bool& finite) {
    using F = Form<FORM>;
    using R = double;
    using SR = typename F::R;   // the storage form's arithmetic type: the values as loaded
    using AT = typename F::AT;
    PopIO<F> io;
    io.hin = static_cast<const typename F::HT*>(a.h);
    io.h0in = static_cast<const float2*>(a.h0);
    io.gin = static_cast<const typename F::GT*>(a.g);
    io.S = a.S; io.hs = SR(C.hs); io.ihs = SR(C.ihs); io.gs = SR(C.gs); io.igs = SR(C.igs);
    const int x = cell % C.nx, y = cell / C.nx;
    const long long c = C.base + cell;
    Nbr<R> nphi, nmu;
    gather(a.tmp_phi, C.nx, C.ny, C.walls, x, y, nphi);
    gather(a.tmp_mu, C.nx, C.ny, C.walls, x, y, nmu);
    Nbr<R> np;
    const AT* pp = static_cast<const AT*>(a.p_prev) + C.base;
    for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
            int yy = y + dy, xx = x + dx;
            xx = xx < 0 ? xx + C.nx : (xx >= C.nx ? xx - C.nx : xx);
            if (C.walls) yy = yy < 0 ? -1 - yy : (yy >= C.ny ? 2 * C.ny - 1 - yy : yy);
            else yy = yy < 0 ? yy + C.ny : (yy >= C.ny ? yy - C.ny : yy);
            np.z[dy + 1][dx + 1] = R(pp[yy * C.nx + xx]);
        }
    R g[9];
    SR hv[9], lo;
    io.phi_of(c, hv, lo);
    finite = isfinite(lo);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        g[i] = R(io.load_g(i, c));   // exact: FP16 or FP32 times a power of two
        finite = finite && isfinite(g[i]) && isfinite(hv[i]);
    }
    R gphix, gphiy, gmux, gmuy, gpx, gpy;
    nphi.grad(gphix, gphiy);
    nmu.grad(gmux, gmuy);
    np.grad(gpx, gpy);
    const R phi = nphi.z[1][1], mu = nmu.z[1][1];
    const Macro<R> m = macroscopic(C, g, phi, mu, gphix, gphiy, gmux, gmuy, nmu.lap(), gpx, gpy);
    // P = p_0 - kappa phi lap(phi) + kappa |grad phi|^2 / 2 + p, p_0 = phi psi' - psi (Sec. 4.2)
    const R psi = C.beta * phi * phi * (phi - R(1)) * (phi - R(1));
    const R dpsi = R(2) * C.beta * phi * (phi - R(1)) * (R(2) * phi - R(1));
    const R Plap = (phi * dpsi - psi) - C.kappa * phi * nphi.lap() +
                   R(0.5) * C.kappa * (gphix * gphix + gphiy * gphiy) + m.p;
    out[0] = phi; out[1] = m.ux; out[2] = m.uy; out[3] = m.p; out[4] = m.rho; out[5] = mu;
    out[6] = Plap;
}

template <int FORM>
__global__ void fields_pass(const AuxArgs a) {
    using R = double;
    Consts<R> C;
    C.load(a.inst[a.instance]);
    const int n = C.nx * C.ny;
    for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < n; cell += gridDim.x * blockDim.x) {
        R v[7];
        bool fin;
        cell_fields<FORM>(a, C, cell, v, fin);
        int k = 0;
        for (int b = 0; b < 7; ++b)
            if (a.mask & (1u << b)) a.out[(long long)(k++) * n + cell] = double(v[b]);
    }
}

// Diagnostics: per-block FP64 partial sums written to a.partials (scratch,
// kDiagBlocks x kDiagQuantities), then one block adds the partials in a fixed
// order, so the result does not depend on timing.
//   0 sum phi, 1 sum rho, 2 kinetic energy, 3 max |u|, 4 sum phi x, 5 sum phi y,
//   6 sum (1-phi) x, 7 sum (1-phi) y, 8 sum P (bulk A), 9 n bulk A,
//   10 sum P (bulk B), 11 n bulk B, 12 non-finite count, 13 sum (1 - phi)
__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

template <int FORM>
__global__ void __launch_bounds__(256) diag_pass(const AuxArgs a) {
    using R = double;
    Consts<R> C;
    C.load(a.inst[a.instance]);
    const int n = C.nx * C.ny;
    double acc[kDiagQuantities];
#pragma unroll
    for (int q = 0; q < kDiagQuantities; ++q) acc[q] = 0.0;
    for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < n; cell += gridDim.x * blockDim.x) {
        R v[7];
        bool fin;
        cell_fields<FORM>(a, C, cell, v, fin);
        const double phi = double(v[0]), ux = double(v[1]), uy = double(v[2]);
        const double rho = double(v[4]), P = double(v[6]);
        const double x = double(cell % C.nx), y = double(cell / C.nx);
        const double uu = ux * ux + uy * uy;
        acc[0] += phi;
        acc[1] += rho;
        acc[2] += 0.5 * rho * uu;
        acc[3] = fmax(acc[3], sqrt(uu));
        acc[4] += phi * x;
        acc[5] += phi * y;
        acc[6] += (1.0 - phi) * x;
        acc[7] += (1.0 - phi) * y;
        if (phi > 1.0 - 1e-3) { acc[8] += P; acc[9] += 1.0; }
        if (phi < 1e-3) { acc[10] += P; acc[11] += 1.0; }
        if (!fin) acc[12] += 1.0;
        acc[13] += 1.0 - phi;
    }
    __shared__ double red[kDiagQuantities][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kDiagQuantities; ++q) {
        const double v = (q == 3) ? warp_max(acc[q]) : warp_sum(acc[q]);
        if (lane == 0) red[q][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < kDiagQuantities) {
        const int q = threadIdx.x;
        double v = red[q][0];
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) v = (q == 3) ? fmax(v, red[q][k]) : v + red[q][k];
        a.partials[blockIdx.x * kDiagQuantities + q] = v;
    }
}

// Final sum of the per-block partials: thread t takes blocks t, t + 256, ...,
// then a fixed shuffle / shared-memory tree combines the threads.
constexpr int kDiagFinalThreads = 256;
static __global__ void __launch_bounds__(kDiagFinalThreads) diag_final(const double* __restrict__ partials,
                                                                       int nblocks, double* __restrict__ result) {
    const int t = threadIdx.x;
    double acc[kDiagQuantities];
#pragma unroll
    for (int q = 0; q < kDiagQuantities; ++q) acc[q] = 0.0;
    for (int b = t; b < nblocks; b += kDiagFinalThreads)
#pragma unroll
        for (int q = 0; q < kDiagQuantities; ++q) {
            const double x = partials[b * kDiagQuantities + q];
            acc[q] = (q == 3) ? fmax(acc[q], x) : acc[q] + x;
        }
    __shared__ double red[kDiagQuantities][kDiagFinalThreads / 32];
    const int lane = t & 31, warp = t >> 5;
#pragma unroll
    for (int q = 0; q < kDiagQuantities; ++q) {
        const double v = (q == 3) ? warp_max(acc[q]) : warp_sum(acc[q]);
        if (lane == 0) red[q][warp] = v;
    }
    __syncthreads();
    if (t < kDiagQuantities) {
        double v = red[t][0];
        for (int w = 1; w < kDiagFinalThreads / 32; ++w) v = (t == 3) ? fmax(v, red[t][w]) : v + red[t][w];
        result[t] = v;
    }
}

template <int FORM>
__global__ void populations_pass(const AuxArgs a, double* out_h, double* out_g) {
    using F = Form<FORM>;
    using R = typename F::R;
    Consts<R> C;
    C.load(a.inst[a.instance]);
    PopIO<F> io;
    io.hin = static_cast<const typename F::HT*>(a.h);
    io.h0in = static_cast<const float2*>(a.h0);
    io.gin = static_cast<const typename F::GT*>(a.g);
    io.S = a.S; io.hs = C.hs; io.ihs = C.ihs; io.gs = C.gs; io.igs = C.igs;
    const int n = C.nx * C.ny;
    for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < n; cell += gridDim.x * blockDim.x) {
        const long long c = C.base + cell;
        for (int i = 0; i < 9; ++i) {
            if (out_h) {
                double v;
                if (F::cons && i == 0) {
                    const float2 h0 = io.load_h0(c);
                    v = double(h0.x) + double(h0.y);
                } else {
                    v = double(io.load_h(i, c));
                }
                out_h[(long long)i * n + cell] = v;
            }
            if (out_g) out_g[(long long)i * n + cell] = double(io.load_g(i, c));
        }
    }
}

}  // namespace lbm
