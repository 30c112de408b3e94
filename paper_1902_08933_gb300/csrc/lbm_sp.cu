// lbm_sp.cu -- the single-phase model of Remark 3 (Sec. 2.3): the generalized
// lattice Boltzmann model with rho~ = rho_0 and a constant density (rho = 1),
// which recovers the incompressible Navier-Stokes equations with a mass source
// (div u = S) and a uniform body force, on the D2Q9 lattice.
//
// One kernel a step, one thread a cell: the cell's populations and source give
// u (Eq. 27a) and p (Eq. 28 with G_0), the equilibrium of Remark 3 (Eq. 25 with
// rho~ = rho_0, rho = 1; g_0 stored shifted by rho_0) and the force term
//   G_i = w_i { S + c_i.F / c_s^2 + (c_i c_i - c_s^2 I):(u F + F u + Q S I) / (2 c_s^4) },
//   Q = (2/d) c_s^2 - xi / (tau_g - 1/2),
// then BGK (Eq. 24) and push-streaming (x periodic; y periodic or halfway
// bounce-back walls). Storage and arithmetic in FP64 or FP32.
#include <cmath>
#include <cstring>
#include <string>

#include "lbm.h"

namespace {

constexpr int kQ = 9;
__host__ __device__ constexpr int sx(int i) { return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0); }
__host__ __device__ constexpr int sy(int i) { return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0); }
__host__ __device__ constexpr double sw(int i) { return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0); }
__host__ __device__ constexpr int sopp(int i) { return i == 0 ? 0 : (i <= 4 ? (i + 1) % 4 + 1 : (i - 5 + 2) % 4 + 5); }
static_assert(sopp(1) == 3 && sopp(2) == 4 && sopp(5) == 7 && sopp(6) == 8 && sopp(8) == 6, "D2Q9 opposites");

struct SpConst {
    int nx, ny, walls;
    double inv_tau, src, tgm, Qc, fx, fy;   // 1/tau_g, 1 - 1/(2 tau_g), tau_g - 1/2, Q, F
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
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
        const R cu = R(sx(i)) * m.ux + R(sy(i)) * m.uy, cF = R(sx(i)) * fx + R(sy(i)) * fy;
        const R c2 = R(sx(i) * sx(i) + sy(i) * sy(i));
        // (c c - c_s^2 I):(u F + F u + Q S I) / (2 c_s^4) = 9 (c.u)(c.F) - 3 u.F + 4.5 (|c|^2 - 2/3) Q S
        G[i] = R(sw(i)) * (S + R(3) * cF + R(9) * cu * cF - R(3) * uF + R(4.5) * (c2 - R(2.0 / 3.0)) * QS);
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
    cudaFree(c->d_tmp);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
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
    if (p.reserved != 0) return LBM_EINVAL;
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
                   1.0 / 3.0 - p.xi / (tau - 0.5), p.force_x, p.force_y};
    const size_t e = sp_elem(precision);
    cudaError_t r;
    if ((r = cudaMalloc(&c->g[0], kQ * c->N * e)) != cudaSuccess ||
        (r = cudaMalloc(&c->g[1], kQ * c->N * e)) != cudaSuccess ||
        (r = cudaMalloc(&c->src, c->N * e)) != cudaSuccess ||
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
    // at rest: p = 0, u = 0, g^eq = rho_0 delta_i0 -- zero with g_0 stored shifted by rho_0
    c->cur = 0;
    if ((r = cudaMemsetAsync(c->g[0], 0, kQ * c->N * sp_elem(c->form), c->stream)) != cudaSuccess)
        return sp_cuda(c, r, "state reset");
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
    for (int s = 0; s < nsteps; ++s) {
        if (c->form == LBM_F64)
            sp_step_kernel<double><<<blocks(c->N), 256, 0, c->stream>>>(
                static_cast<const double*>(c->g[c->cur]), static_cast<double*>(c->g[1 - c->cur]),
                static_cast<const double*>(c->src), c->N, c->K);
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
    const unsigned ok = LBM_FIELD_UX | LBM_FIELD_UY | LBM_FIELD_P;
    if (!host_out || mask == 0 || (mask & ~ok)) return sp_fail(c, LBM_EINVAL, "bad mask or output");
    if (!c->ready) return sp_fail(c, LBM_ESTATE, "not initialised");
    const int nf = ((mask & LBM_FIELD_UX) ? 1 : 0) + ((mask & LBM_FIELD_UY) ? 1 : 0) + ((mask & LBM_FIELD_P) ? 1 : 0);
    if (c->form == LBM_F64)
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
    if (c->form == LBM_F64)
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
