// lbm_step_tma.cuh -- the fused step kernel fed by the Tensor Memory Accelerator.
//
// Same arithmetic and the same row march as step_kernel (lbm_device.cuh), but the
// global loads of each row leave the computing threads: one thread issues bulk
// asynchronous copies (cp.async.bulk, global -> shared, completion counted in
// bytes on an mbarrier) of the next row's data one row ahead, so the copies of
// row Y + 1 are in flight while row Y is collided.
//
// Copies of packet k + 1 are issued, one per lane of the last warp, after the
// first barrier of iteration k (every thread is then past the collision of the
// previous row, so the stages being refilled are no longer read).
//
// Packet k (row Y_k = ystart + k d of the march) carries
//   h  of the lead row Y_k + 2d  (9 planes; 16-byte halo chunks on both sides),
//   p  of row Y_k + d            (previous step's pressure, halo chunks),
//   g  and phi*u of row Y_k      (collision row, strip only).
// h/p packets live in 4 stages (read at iteration k for phi, at k+2 for the
// collision; p at k, k+1, k+2); g packets in 2 stages. Packets -2 and -1 (h/p
// only) prime the march. Used only when every copy is 16-byte aligned:
// nx % 8 == 0 (rows of every storage type start on 16 bytes) -- the host checks.
//
// Every wait on an mbarrier is bounded. If one runs out, the block agrees on it
// (__syncthreads_or), writes LBM_ETIMEOUT to the status word, waits (bounded)
// for the copies it issued and leaves; the host reports the status.
#pragma once

#include <type_traits>

#include "lbm_device.cuh"
#include "lbm_mbar.cuh"

namespace lbm {

// Halo chunk: 16 bytes of a plane row, the smallest aligned bulk copy.
template <typename T> struct Halo { static constexpr int n = 16 / (int)sizeof(T); };

// Shared-memory layout of the TMA kernel (bytes, every segment 16-byte aligned).
template <int FORM, int TX>
struct TmaSmem {
    using F = Form<FORM>;
    using R = typename F::R;
    using HT = typename F::HT;
    using GT = typename F::GT;
    using AT = typename F::AT;
    static constexpr int HH = Halo<HT>::n, HA = Halo<AT>::n, H0 = Halo<float2>::n;
    static constexpr int PW = TX + 4, MW = TX + 2;
    static constexpr size_t h0seg = F::cons ? (size_t)(TX + 2 * H0) * sizeof(float2) : 0;
    static constexpr size_t hseg = (size_t)(TX + 2 * HH) * sizeof(HT);
    static constexpr int hplanes = F::cons ? 8 : 9;
    static constexpr size_t pseg = (size_t)(TX + 2 * HA) * sizeof(AT);
    static constexpr size_t hp_stage = h0seg + hplanes * hseg + pseg;
    static constexpr size_t g_stage = 9 * (size_t)TX * sizeof(GT) + 2 * (size_t)TX * sizeof(AT);
    static constexpr int NSH = 4, NSG = 2;
    static constexpr size_t off_hp = 0;
    static constexpr size_t off_g = off_hp + NSH * hp_stage;
    static constexpr size_t off_phi = off_g + NSG * g_stage;
    static constexpr size_t off_mu = off_phi + 8 * PW * sizeof(R);
    static constexpr size_t off_lo = off_mu + 4 * MW * sizeof(R);            // phi low parts
    static constexpr size_t off_bar = (off_lo + (F::cons ? 4 * TX * sizeof(R) : 0) + 15) / 16 * 16;
    static constexpr size_t bytes = off_bar + (NSH + NSG) * 8;
    static_assert(hseg % 16 == 0 && pseg % 16 == 0 && h0seg % 16 == 0, "segments must stay aligned");
    static_assert(hp_stage % 16 == 0 && g_stage % 16 == 0, "stages must stay aligned");
};

template <int FORM, int TX>
struct TmaOcc {   // register budget: FP32 forms, 5 blocks of 128 threads (smem-bound anyway)
    static constexpr int value = (640 / TX) > 0 ? 640 / TX : 1;
};

template <int FORM, int TX>
__global__ void __launch_bounds__(TX, TmaOcc<FORM, TX>::value) step_kernel_tma(const StepArgs a) {
    using F = Form<FORM>;
    using R = typename F::R;
    using HT = typename F::HT;
    using GT = typename F::GT;
    using AT = typename F::AT;
    using L = TmaSmem<FORM, TX>;
    static_assert(sizeof(R) == 4, "the TMA-fed kernel serves the FP32-arithmetic forms");
    constexpr int PW = L::PW, MW = L::MW, HH = L::HH, HA = L::HA, H0 = L::H0;
    extern __shared__ __align__(128) unsigned char smem[];
    R* phiR = reinterpret_cast<R*>(smem + L::off_phi);     // [8][PW]
    R* muR = reinterpret_cast<R*>(smem + L::off_mu);       // [4][MW]
    R* loR = reinterpret_cast<R*>(smem + L::off_lo);       // [4][TX] (conservative forms)
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::off_bar);

    const WorkItem wk = a.work[blockIdx.x];
    Consts<R> C;
    C.load(a.inst[wk.inst]);
    const int nx = C.nx, ny = C.ny, walls = C.walls;
    const int x0 = wk.x0, d = wk.dir;
    const int w = min(TX, nx - x0);
    const int tid = threadIdx.x;
    const int base = (int)C.base;
    const long long S = a.S;
    const HT* hin = static_cast<const HT*>(a.h_in);
    const float2* h0in = static_cast<const float2*>(a.h0_in);
    const GT* gin = static_cast<const GT*>(a.g_in);
    const AT* p_in = static_cast<const AT*>(a.p_in);
    AT* phiu = static_cast<AT*>(a.phiu);
    PopIO<F> io;
    io.hin = hin;
    io.hout = static_cast<HT*>(a.h_out);
    io.h0in = h0in;
    io.h0out = static_cast<float2*>(a.h0_out);
    io.gin = gin;
    io.gout = static_cast<GT*>(a.g_out);
    io.S = S; io.hs = C.hs; io.ihs = C.ihs; io.gs = C.gs; io.igs = C.igs;
    AT* p_out = static_cast<AT*>(a.p_out);

    auto wrapx = [nx](int x) { return x < 0 ? x + nx : (x >= nx ? x - nx : x); };
    auto rowg = [ny, walls](int y) { return walls ? y : (y < 0 ? y + ny : (y >= ny ? y - ny : y)); };
    auto ghost = [ny, walls](int y) { return walls && (y < 0 || y >= ny); };
    auto mirror = [ny](int y) { return y < 0 ? -1 - y : 2 * ny - 1 - y; };
    auto rowoff = [&](int y) { return base + rowg(y) * nx; };

    // stage accessors
    auto hp_stage = [&](int j) { return smem + L::off_hp + (size_t)((j + 2) & 3) * L::hp_stage; };
    auto g_stage = [&](int j) { return smem + L::off_g + (size_t)(j & 1) * L::g_stage; };
    auto hbar = [&](int j) { return smem_u32(&bars[(j + 2) & 3]); };
    auto gbar = [&](int j) { return smem_u32(&bars[L::NSH + (j & 1)]); };
    auto hpar = [](int j) { return (uint32_t)(((j + 2) >> 2) & 1); };
    auto gpar = [](int j) { return (uint32_t)((j >> 1) & 1); };

    // ---- producer: the last warp queues the ~41 copies of packet j, one per lane
    // (lane 0 first announces the byte counts on the two mbarriers).
    auto issue = [&](int j, int lane) {
        const int Yj = wk.ystart + j * d;
        const int Lr = Yj + 2 * d, Mr = Yj + d;
        const bool lead = !ghost(Lr);
        const int xl = x0 == 0 ? nx : x0;             // left halo chunk ends at xl (wrapped)
        const int xr = x0 + w == nx ? 0 : x0 + w;     // right halo chunk starts at xr (wrapped)
        const uint32_t hb = hbar(j), gb = gbar(j);
        const uint32_t st = smem_u32(hp_stage(j));
        const uint32_t gs = smem_u32(g_stage(j));
        if (lane == 0) {
            uint32_t hp_bytes = (uint32_t)((w + 2 * HA) * sizeof(AT));
            if (lead) {
                hp_bytes += (uint32_t)(L::hplanes * (size_t)(w + 2 * HH) * sizeof(HT));
                if constexpr (F::cons) hp_bytes += (uint32_t)((w + 2 * H0) * sizeof(float2));
            }
            mbar_expect_tx(hb, hp_bytes);
            if (j >= 0) mbar_expect_tx(gb, (uint32_t)(9 * w * sizeof(GT) + 2 * w * sizeof(AT)));
        }
        __syncwarp();
        const int roL = lead ? rowoff(Lr) : 0;
        const int roM = base + (ghost(Mr) ? mirror(Mr) : rowg(Mr)) * nx;
        const int roY = rowoff(Yj) + x0;
        // copy c: 0..26 h (plane c / 3, part c % 3), 27..29 p, 30..38 g, 39..40 phi*u
        for (int c = lane; c < 41; c += 32) {
            const char* src;
            uint32_t dst, bytes;
            uint32_t bar = hb;
            if (c < 30) {
                if (c < 27 && !lead) continue;
                const int plane = c < 27 ? c / 3 : -1, part = c % 3;
                int es, hh;
                const char* row;
                uint32_t seg;
                if (plane < 0) {                                   // pressure row
                    es = (int)sizeof(AT); hh = HA;
                    row = reinterpret_cast<const char*>(p_in + roM);
                    seg = st + (uint32_t)(L::h0seg + L::hplanes * L::hseg);
                } else if (F::cons && plane == 0) {                // h_0 pair plane
                    es = (int)sizeof(float2); hh = H0;
                    row = reinterpret_cast<const char*>(h0in + roL);
                    seg = st;
                } else {
                    const int pl = F::cons ? plane - 1 : plane;
                    es = (int)sizeof(HT); hh = HH;
                    row = reinterpret_cast<const char*>(hin + pl * S + roL);
                    seg = st + (uint32_t)(L::h0seg + pl * L::hseg);
                }
                const int col = part == 0 ? xl - hh : (part == 1 ? x0 : xr);
                src = row + (long long)col * es;
                dst = seg + (uint32_t)(part == 0 ? 0 : (part == 1 ? hh * es : (hh + w) * es));
                bytes = (uint32_t)((part == 1 ? w : hh) * es);
            } else {
                if (j < 0) break;
                bar = gb;
                if (c < 39) {
                    const int i = c - 30;
                    src = reinterpret_cast<const char*>(gin + i * S + roY);
                    dst = gs + (uint32_t)(i * TX * sizeof(GT));
                    bytes = (uint32_t)(w * sizeof(GT));
                } else {
                    const int i = c - 39;
                    src = reinterpret_cast<const char*>(phiu + i * S + roY);
                    dst = gs + (uint32_t)(9 * TX * sizeof(GT) + i * TX * sizeof(AT));
                    bytes = (uint32_t)(w * sizeof(AT));
                }
            }
            bulk_load(dst, src, bytes, bar, a.status);
        }
    };

    // ---- stage readers
    // h_i of packet j at strip column s (x = x0 - 2 + s), 1 <= i <= 8 for conservative forms
    auto st_h = [&](int j, int i, int s) -> R {
        const unsigned char* st = hp_stage(j) + L::h0seg;
        const int pl = F::cons ? i - 1 : i;
        const HT* seg = reinterpret_cast<const HT*>(st + pl * L::hseg);
        if constexpr (F::h16) return ldr<HT, R>(seg + (HH - 2 + s)) * C.ihs;
        else return ldr<HT, R>(seg + (HH - 2 + s));
    };
    auto st_h0 = [&](int j, int s) -> float2 {
        return reinterpret_cast<const float2*>(hp_stage(j))[H0 - 2 + s];
    };
    auto st_p = [&](int j, int s) -> R {   // p column x0 - 1 + s
        const AT* seg = reinterpret_cast<const AT*>(hp_stage(j) + L::h0seg + L::hplanes * L::hseg);
        return R(seg[HA - 1 + s]);
    };
    auto phi_at = [&](int j, int s, R hv[9], R& lo) -> R {
        if constexpr (F::cons) {
            R s8 = R(0);
#pragma unroll
            for (int i = 1; i < 9; ++i) { hv[i] = st_h(j, i, s); s8 += hv[i]; }
            const float2 h0 = st_h0(j, s);
            float sm, e, hi, l2;
            two_sum(h0.x, s8, sm, e);
            fast_two_sum(sm, e + h0.y, hi, l2);
            hv[0] = hi - s8;
            lo = l2;
            return hi;
        } else {
#pragma unroll
            for (int i = 0; i < 9; ++i) hv[i] = st_h(j, i, s);
            R phi = hv[0];
#pragma unroll
            for (int i = 1; i < 9; ++i) phi += hv[i];
            lo = R(0);
            return phi;
        }
    };

    const bool lead0 = tid < w + 4, lead1 = tid + TX < w + 4;
    const bool mid0 = tid < w + 2, mid1 = tid + TX < w + 2;
    const bool act = tid < w;
    const int X = x0 + tid;
    const int colm = act ? wrapx(X - 1) : 0, colp = act ? wrapx(X + 1) : 0;

    // phi of row Lr from packet j (j = -2, -1, ...) or, for ghost rows, the mirror
    auto lead_from_packet = [&](int j, int Lr) {
        R* prow = phiR + ((Lr + 64) & 7) * PW;
        if (ghost(Lr)) {
            const R* src = phiR + ((mirror(Lr) + 64) & 7) * PW;
            if (lead0) prow[tid] = src[tid];
            if (lead1) prow[tid + TX] = src[tid + TX];
            return;
        }
        auto column = [&](int s) {
            R hv[9], lo;
            prow[s] = phi_at(j, s, hv, lo);
            if constexpr (F::cons) {
                if (s >= 2 && s < w + 2) loR[((Lr + 64) & 3) * TX + (s - 2)] = lo;
            }
        };
        if (lead0) column(tid);
        if (lead1) column(tid + TX);
    };
    // phi of row Lr straight from global memory (the two prologue rows behind Y0)
    auto lead_from_global = [&](int Lr) {
        R* prow = phiR + ((Lr + 64) & 7) * PW;
        const int ro = rowoff(Lr);
        auto column = [&](int s) {
            R hv[9], lo;
            prow[s] = io.phi_of(ro + wrapx(x0 - 2 + s), hv, lo);
        };
        if (lead0) column(tid);
        if (lead1) column(tid + TX);
    };
    auto ghost_copy = [&](int Lr) {
        R* prow = phiR + ((Lr + 64) & 7) * PW;
        const R* src = phiR + ((mirror(Lr) + 64) & 7) * PW;
        if (lead0) prow[tid] = src[tid];
        if (lead1) prow[tid + TX] = src[tid + TX];
    };
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
    auto collide_row = [&](int k) {
        if (!act) return;
        const int Y = wk.ystart + k * d;
        const int rY = rowoff(Y);
        const int c = rY + X;
        Nbr<R> nphi, nmu, np;
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
            const R* pr = phiR + ((Y + dy - 1 + 64) & 7) * PW + tid + 1;
            const R* mr = muR + ((Y + dy - 1 + 64) & 3) * MW + tid;
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
                nphi.z[dy][dx] = pr[dx];
                nmu.z[dy][dx] = mr[dx];
            }
        }
        // p of rows Y - 1, Y, Y + 1 sit in packets k - 2, k - 1, k (rows Y - d, Y, Y + d)
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
            const R pm = st_p(k - 2, tid + dx), p0 = st_p(k - 1, tid + dx), pp = st_p(k, tid + dx);
            np.z[1][dx] = p0;
            np.z[0][dx] = d > 0 ? pm : pp;
            np.z[2][dx] = d > 0 ? pp : pm;
        }
        const R phi = nphi.z[1][1], mu = nmu.z[1][1];
        R gphix, gphiy, gmux, gmuy, gpx, gpy;
        nphi.grad(gphix, gphiy);
        nmu.grad(gmux, gmuy);
        np.grad(gpx, gpy);
        const R lapmu = nmu.lap();
        R h[9], g[9];
        // h of row Y = lead row of packet k - 2
#pragma unroll
        for (int i = F::cons ? 1 : 0; i < 9; ++i) h[i] = st_h(k - 2, i, tid + 2);
        if constexpr (F::cons) h[0] = loR[((Y + 64) & 3) * TX + tid];
        const unsigned char* gs = g_stage(k);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const GT* gp = reinterpret_cast<const GT*>(gs + (size_t)i * TX * sizeof(GT));
            g[i] = F::g16 ? ldr<GT, R>(gp + tid) * C.igs : ldr<GT, R>(gp + tid);
        }
        const AT* pu = reinterpret_cast<const AT*>(gs + 9 * (size_t)TX * sizeof(GT));
        const R pux = R(pu[tid]), puy = R(pu[TX + tid]);

        const Macro<R> m = macroscopic(C, g, phi, mu, gphix, gphiy, gmux, gmuy, lapmu, gpx, gpy);
        const R phiux = phi * m.ux, phiuy = phi * m.uy;
        R gpost[9], hpost[9];
        collide_cell(C, m, phi, mu, phiux - pux, phiuy - puy, g, h, gpost, hpost);
        float2 h0c = make_float2(0.f, 0.f);
        if constexpr (F::cons) {
            R rest = R(0);
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                hpost[i] = io.round_h(hpost[i]);
                rest += hpost[i];
            }
            h0c = io.conservative_h0(phi, h[0], rest);
        }
        const bool bot = walls && Y == 0, top = walls && Y == ny - 1;
        const int rDn = bot ? 0 : rowoff(Y - 1);
        const int rUp = top ? 0 : rowoff(Y + 1);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int cyi = cy_of(i), cxi = cx_of(i);
            const int col = cxi < 0 ? colm : (cxi > 0 ? colp : X);
            int dst = (cyi == 0 ? rY : (cyi > 0 ? rUp : rDn)) + col;
            int kk = i;
            if ((cyi > 0 && top) || (cyi < 0 && bot)) {
                dst = c;
                kk = opp_of(i);
            }
            if constexpr (F::cons) {
                if (i == 0) io.store_h0(dst, h0c);
                else io.store_h(kk, dst, hpost[i]);
            } else {
                io.store_h(kk, dst, hpost[i]);
            }
            io.store_g(kk, dst, gpost[i]);
        }
        phiu[c] = AT(phiux);
        phiu[S + c] = AT(phiuy);
        p_out[c] = AT(m.p);
    };

    // bounded wait for packet j's copies by every thread; true if all arrived
    auto wait_packet = [&](int j) {
        bool ok = mbar_wait(hbar(j), hpar(j));
        if (j >= 0) ok = mbar_wait(gbar(j), gpar(j)) && ok;
        return ok;
    };
    auto bail = [&](int first, int last) {   // copies of packets first..last may be in flight
        if (tid == 0) {
            atomicExch(a.status, kStatusTimeout);
            for (int j = first; j <= last; ++j) wait_packet(j);
        }
    };

    // ---- prologue
    const int warp = tid >> 5, lane = tid & 31;
    const bool producer = warp == TX / 32 - 1;
    if (tid == 0) {
        for (int b = 0; b < L::NSH + L::NSG; ++b) mbar_init(smem_u32(&bars[b]), 1);
        fence_mbar_init();
        fence_proxy_async();
    }
    __syncthreads();
    if (producer) {
        issue(-2, lane);
        issue(-1, lane);
        issue(0, lane);
    }
    const int Y0 = wk.ystart;
    {
        const bool ok = wait_packet(-2) && wait_packet(-1);
        if (__syncthreads_or(!ok)) { bail(-2, 0); return; }
    }
    // phi rows: inside the domain first, ghosts (mirror copies) after
    lead_from_packet(-2, Y0);                                   // never a ghost
    if (!ghost(Y0 + d)) lead_from_packet(-1, Y0 + d);
    if (!ghost(Y0 - d)) lead_from_global(Y0 - d);
    if (!ghost(Y0 - 2 * d)) lead_from_global(Y0 - 2 * d);
    if (ghost(Y0 + d)) ghost_copy(Y0 + d);
    if (ghost(Y0 - d)) ghost_copy(Y0 - d);
    if (ghost(Y0 - 2 * d)) ghost_copy(Y0 - 2 * d);
    __syncthreads();
    mu_row(Y0);
    mu_row(Y0 - d);
    __syncthreads();

    for (int k = 0; k < wk.nrows; ++k) {
        const int Y = Y0 + k * d;
        // A: phi of the lead row from packet k (every thread waits for it itself)
        const bool ok = wait_packet(k);
        lead_from_packet(k, Y + 2 * d);
        // the barrier also tells every thread whether a wait ran out
        if (__syncthreads_or(!ok)) { bail(k, k); return; }
        // all threads are past the collision of row Y - d: the stages of packets
        // k - 3 (h/p) and k - 1 (g) are free for packet k + 1
        if (producer && k + 1 < wk.nrows) {
            if (lane == 0) fence_proxy_async();
            __syncwarp();
            issue(k + 1, lane);
        }
        mu_row(Y + d);                     // B
        __syncthreads();
        collide_row(k);                    // C
    }
}

}  // namespace lbm
