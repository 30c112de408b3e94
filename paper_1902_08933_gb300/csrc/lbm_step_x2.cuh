// lbm_step_x2.cuh -- the fused step kernel with two cells per thread.
//
// Same row march and arithmetic as step_kernel (lbm_device.cuh) for the FP32
// forms, but every thread owns two horizontally adjacent cells (X, X+1), X even,
// and computes them together in the two lanes of the packed FP32 instructions of
// sm_100+ (FFMA2 / FADD2 / FMUL2 through the F2 value type). A pair is one 8-byte
// (FP32) or 4-byte (FP16) element in memory, so the loads of g, h, phi*u and p
// and the stores that keep the pair together (directions with c_x = 0) are
// vector accesses; the shared-memory stencils read three 8-byte words per row.
// Per cell this halves the address arithmetic, the per-row bookkeeping and the
// floating-point instruction count of the collision.
//
// Rings in shared memory, each row RW = 2 TX + 8 entries, column x at index
// x - x0 + 4 (even columns on 8-byte boundaries; the outer two entries on each
// side are padding that only ever feeds values nobody reads):
//   phi [8][RW], mu [4][RW], p [4][RW] (FP32), and 4 slots of h in its storage
//   type: [RW] (hi, lo) pairs of the conservative h_0, then the planes.
// Loads of the lead row (h) and of the p row run ahead: each thread copies its
// own column pairs of the next iteration's rows with cp.async right after the
// first barrier of the iteration, and waits only for its own copies at the next
// phase A (the same schedule as step_kernel<..., true>).
// Requires nx even (a pair never straddles the periodic seam); the host checks.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

__device__ __forceinline__ F2 ld_pair(const float* p) { return F2(*reinterpret_cast<const float2*>(p)); }
__device__ __forceinline__ F2 ld_pair(const __half* p) {
    return F2(__half22float2(*reinterpret_cast<const __half2*>(p)));
}
__device__ __forceinline__ void st_pair(float* p, F2 v) { *reinterpret_cast<float2*>(p) = v.v; }
__device__ __forceinline__ void st_pair(__half* p, F2 v) {
    *reinterpret_cast<__half2*>(p) = __float22half2_rn(v.v);
}
__device__ __forceinline__ F2 lds_pair(const float* p) { return F2(*reinterpret_cast<const float2*>(p)); }
// The two cells' results in the storage type of a plane (FP16: one packed
// conversion for both), then stored as a pair or one cell at a time.
__device__ __forceinline__ float2 to_store(F2 v, const float*) { return v.v; }
__device__ __forceinline__ __half2 to_store(F2 v, const __half*) { return __float22half2_rn(v.v); }
__device__ __forceinline__ void st_both(float* p, float2 v) { *reinterpret_cast<float2*>(p) = v; }
__device__ __forceinline__ void st_both(__half* p, __half2 v) { *reinterpret_cast<__half2*>(p) = v; }
__device__ __forceinline__ void st_first(float* p, float2 v) { *p = v.x; }
__device__ __forceinline__ void st_first(__half* p, __half2 v) { *p = __low2half(v); }
__device__ __forceinline__ void st_second(float* p, float2 v) { *p = v.y; }
__device__ __forceinline__ void st_second(__half* p, __half2 v) { *p = __high2half(v); }
// the stored values read back as FP32 (exact)
__device__ __forceinline__ float first_f(float2 v) { return v.x; }
__device__ __forceinline__ float first_f(__half2 v) { return __low2float(v); }
__device__ __forceinline__ float second_f(float2 v) { return v.y; }
__device__ __forceinline__ float second_f(__half2 v) { return __high2float(v); }

template <int FORM, int TX>
struct X2Smem {
    using F = Form<FORM>;
    using HT = typename F::HT;
    static constexpr int SW = 2 * TX;   // strip width in columns
    static constexpr int RW = SW + 8;
    static constexpr size_t H0B = F::cons ? (size_t)RW * sizeof(float2) : 0;   // h_0 pairs (hi, lo)
    static constexpr size_t HPB = (size_t)RW * sizeof(HT);                      // one plane, storage type
    static constexpr size_t SLOT = H0B + (F::cons ? 8 : 9) * HPB;
    static constexpr size_t RINGS = (size_t)(8 * RW + 4 * RW + 4 * RW) * sizeof(float);
    static constexpr size_t bytes = RINGS + 4 * SLOT;
    static_assert(SLOT % 16 == 0 && RINGS % 16 == 0, "h slots must stay 16-byte aligned");
};

// Resident blocks per SM the kernel is compiled for. Measured on the 1024 x 4096
// bubble: 384 / TX blocks (up to 168 registers a thread) beat 512 / TX (128
// registers) by 17 % for FP32 storage -- the extra registers let the loads of
// the collision row fly longer -- while the FP16-h form, with half the bytes
// a cell to wait for, is faster with the fourth block. Never more blocks than
// the shared-memory rings allow (228 KB a SM, 1 KB of it reserved per block).
template <int FORM, int TX>
struct X2Occ {
    static constexpr int by_regs = ((Form<FORM>::h16 ? 512 : 384) / TX) > 0 ? (Form<FORM>::h16 ? 512 : 384) / TX : 1;
    static constexpr int by_smem = (int)((228u * 1024u) / (X2Smem<FORM, TX>::bytes + 1024u));
    static constexpr int value = by_smem < 1 ? 1 : (by_smem < by_regs ? by_smem : by_regs);
};

// One work item (a strip of 2 TX columns of one instance, a run of rows) marched
// by a group of TX threads (32, 64 or 128): a whole thread block (step_kernel_x2:
// barrier 0, the one __syncthreads uses; TX its compile-time block size, so the
// layout below folds to constants) or a thread group of the batched kernel
// (step_kernel_x2_batched: named barrier 1 + group, TX 128 or 64 chosen per block
// descriptor). smem_raw is the group's own region in the X2Smem<FORM, TX> layout,
// tid the thread's index in the group, item the work item's index in
// StepArgs::work (and of its monitor slot); swap: the step reads the *_out
// buffers of a and writes the *_in ones (odd steps of a batched launch).
template <int FORM, int MON>
__device__ __forceinline__ void x2_item(const StepArgs& a, int item, unsigned char* smem_raw, int tid,
                                        int bar, int grp, const int TX, const bool swap = false,
                                        const int step = 0) {
    using F = Form<FORM>;
    using HT = typename F::HT;
    using GT = typename F::GT;
    static_assert(sizeof(typename F::R) == 4, "the paired kernel serves the FP32-arithmetic forms");
    // X2Smem<FORM, TX>'s layout for this group width
    const int SW = 2 * TX, RW = SW + 8;
    const size_t H0B = F::cons ? (size_t)RW * sizeof(float2) : 0;
    const size_t HPB = (size_t)RW * sizeof(HT);
    const size_t SLOT = H0B + (F::cons ? 8 : 9) * HPB;
    float* phiR = reinterpret_cast<float*>(smem_raw);   // [8][RW]
    float* muR = phiR + 8 * RW;                          // [4][RW]
    float* pR = muR + 4 * RW;                            // [4][RW]
    unsigned char* hR = smem_raw + (size_t)16 * RW * sizeof(float);   // [4] slots of SLOT bytes

    const WorkItem wk = a.work[item];
    Consts<float> C;
    C.load(a.inst[wk.inst]);
    const int nx = C.nx, ny = C.ny, walls = C.walls;
    const int x0 = wk.x0, d = wk.dir;
    const int w = min(SW, nx - x0);
    const int base = (int)C.base;
    const long long S = a.S;
    // the two buffer sets lie set_delta bytes apart, every array at the same
    // offset in both: a swapped step moves all the pointers by that one amount
    const long long sw = swap ? a.set_delta : 0;
    auto moved = [sw](const void* p, long long sign) {
        return static_cast<const void*>(static_cast<const char*>(p) + sign * sw);
    };
    const HT* hin = static_cast<const HT*>(moved(a.h_in, 1));
    HT* hout = static_cast<HT*>(const_cast<void*>(moved(a.h_out, -1)));
    const float2* h0in = static_cast<const float2*>(moved(a.h0_in, 1));
    float2* h0out = static_cast<float2*>(const_cast<void*>(moved(a.h0_out, -1)));
    const GT* gin = static_cast<const GT*>(moved(a.g_in, 1));
    GT* gout = static_cast<GT*>(const_cast<void*>(moved(a.g_out, -1)));
    const float* p_in = static_cast<const float*>(moved(a.p_in, 1));
    float* p_out = static_cast<float*>(const_cast<void*>(moved(a.p_out, -1)));
    float* phiu = static_cast<float*>(a.phiu);
    // FP16 planes hold their values times a power-of-two scale (hs, gs); the
    // arithmetic keeps h and g in those units (collide_emit / macroscopic with
    // their scale flags), so only the sum of h that forms phi is un-scaled.
    const float ihs = C.ihs;
    MonAcc<F2> mon;

    auto wrapx = [nx](int x) { return x < 0 ? x + nx : (x >= nx ? x - nx : x); };
    auto rowg = [ny, walls](int y) { return walls ? y : (y < 0 ? y + ny : (y >= ny ? y - ny : y)); };
    auto ghost = [ny, walls](int y) { return walls && (y < 0 || y >= ny); };
    auto mirror = [ny](int y) { return y < 0 ? -1 - y : 2 * ny - 1 - y; };
    auto rowoff = [&](int y) { return base + rowg(y) * nx; };
    auto prow = [&](int y) { return phiR + ((y + 64) & 7) * RW; };
    auto mrow = [&](int y) { return muR + ((y + 64) & 3) * RW; };
    auto qrow = [&](int y) { return pR + ((y + 64) & 3) * RW; };
    auto hslot = [&](int y) { return hR + ((y + 64) & 3) * SLOT; };
    // plane i (i >= 1 for conservative forms) of the h slot of row y, storage type
    auto hplane = [&](int y, int i) {
        return reinterpret_cast<HT*>(hslot(y) + H0B + (F::cons ? i - 1 : i) * HPB);
    };
    auto hpairs = [&](int y) { return reinterpret_cast<float2*>(hslot(y)); };   // conservative h_0
    // population i of the cell pair at c as stored (FP16: still scaled by gs)
    auto ld_g = [&](int i, int c) -> F2 { return ld_pair(gin + (long long)i * S + c); };
    // output planes: h_k (k >= 1 for conservative forms), g_k
    auto hplane_out = [&](int k) { return hout + (long long)(F::cons ? k - 1 : k) * S; };
    auto gplane_out = [&](int k) { return gout + (long long)k * S; };

    // Column pairs of the lead / p rows: pair q covers x0-2+2q, x0-1+2q (ring index 2+2q).
    const int nq = (w + 4) >> 1;
    const bool q0 = tid < nq, q1 = tid + TX < nq;
    const int qc0 = q0 ? wrapx(x0 - 2 + 2 * tid) : 0;
    const int qc1 = q1 ? wrapx(x0 - 2 + 2 * (tid + TX)) : 0;
    // The collision pair of this thread.
    const bool act = 2 * tid < w;
    const int X = x0 + 2 * tid;
    const int jX = 2 * tid + 4;
    const int colm = act ? wrapx(X - 1) : 0, colp = act ? wrapx(X + 2) : 0;

    // phi of the pair at ring index j of row Lr from the raw values in its h slot
    // (conservative forms: the low part of phi goes back into the h_0 pair slot)
    auto phi_from_slot = [&](int Lr, int j) {
        F2 phi;
        if constexpr (F::cons) {
            F2 s8 = F2(0.f);
#pragma unroll
            for (int i = 1; i < 9; ++i) s8 = s8 + ld_pair(hplane(Lr, i) + j);
            if constexpr (F::h16) s8 = s8 * ihs;   // exact: ihs is a power of two
            float4* h0p = reinterpret_cast<float4*>(&hpairs(Lr)[j]);
            const float4 h0 = *h0p;                                     // (hi, lo) of both cells
            float sa, ea, ha, la, sb, eb, hb, lb;
            two_sum(h0.x, s8.v.x, sa, ea);
            fast_two_sum(sa, ea + h0.y, ha, la);
            two_sum(h0.z, s8.v.y, sb, eb);
            fast_two_sum(sb, eb + h0.w, hb, lb);
            phi = F2(ha, hb);
            *h0p = make_float4(0.f, la, 0.f, lb);                       // low parts of phi
        } else {
            static_assert(!F::h16, "FP16 h is stored with the conservative h_0 only");
            phi = ld_pair(hplane(Lr, 0) + j);
#pragma unroll
            for (int i = 1; i < 9; ++i) phi = phi + ld_pair(hplane(Lr, i) + j);   // Eq. 18
        }
        st_pair(prow(Lr) + j, phi);
    };
    // A (synchronous, prologue). Pair q of row Lr: copy the stored values into the
    // slot, then phi.
    auto lead_pair = [&](int Lr, int q, int col) {
        const int c = rowoff(Lr) + col;
        const int j = 2 + 2 * q;
        if constexpr (F::cons)
            *reinterpret_cast<float4*>(&hpairs(Lr)[j]) = *reinterpret_cast<const float4*>(h0in + c);
#pragma unroll
        for (int i = F::cons ? 1 : 0; i < 9; ++i) {
            const HT* src = hin + (long long)(F::cons ? i - 1 : i) * S + c;
            if constexpr (F::h16) *reinterpret_cast<__half2*>(hplane(Lr, i) + j) = *reinterpret_cast<const __half2*>(src);
            else *reinterpret_cast<float2*>(hplane(Lr, i) + j) = *reinterpret_cast<const float2*>(src);
        }
        phi_from_slot(Lr, j);
    };
    auto ghost_row = [&](int Lr) {   // mirror ghost row next to a wall (reading Q7)
        float* dst = prow(Lr);
        const float* src = prow(mirror(Lr));
        if (q0) st_pair(dst + 2 + 2 * tid, lds_pair(src + 2 + 2 * tid));
        if (q1) st_pair(dst + 2 + 2 * (tid + TX), lds_pair(src + 2 + 2 * (tid + TX)));
    };
    auto lead_row = [&](int Lr) {
        if (ghost(Lr)) { ghost_row(Lr); return; }
        if (q0) lead_pair(Lr, tid, qc0);
        if (q1) lead_pair(Lr, tid + TX, qc1);
    };
    // Asynchronous copies of this thread's column pairs of lead row Lr and p row M.
    auto prefetch = [&](int Lr, int M) {
        auto h_pair = [&](int q, int col) {
            const int c = rowoff(Lr) + col;
            const int j = 2 + 2 * q;
            if constexpr (F::cons) cp_async16(&hpairs(Lr)[j], h0in + c);
#pragma unroll
            for (int i = F::cons ? 1 : 0; i < 9; ++i) {
                const HT* src = hin + (long long)(F::cons ? i - 1 : i) * S + c;
                if constexpr (F::h16) cp_async4(hplane(Lr, i) + j, src);
                else cp_async8(hplane(Lr, i) + j, src);
            }
        };
        if (!ghost(Lr)) {
            if (q0) h_pair(tid, qc0);
            if (q1) h_pair(tid + TX, qc1);
        }
        const float* src = p_in + base + (ghost(M) ? mirror(M) : rowg(M)) * nx;
        float* dst = qrow(M);
        if (q0) cp_async8(dst + 2 + 2 * tid, src + qc0);
        if (q1) cp_async8(dst + 2 + 2 * (tid + TX), src + qc1);
        cp_async_commit();
    };
    // L2 prefetch of the g and phi*u row segments of collision row Yp (the next
    // one): eleven bulk prefetches (cp.async.bulk.prefetch.L2, sm_90+), one a
    // lane, over the 16-byte-aligned interior of each segment. A hint only: no
    // completion to wait for; the collision's own loads then hit L2.
    auto l2_prefetch_row = [&](int Yp) {
        if (tid >= 11 || ghost(Yp)) return;
        const long long c = (long long)rowoff(Yp) + x0;
        const char* src;
        unsigned bytes;
        if (tid < 9) {
            src = reinterpret_cast<const char*>(gin + (long long)tid * S + c);
            bytes = (unsigned)(w * sizeof(GT));
        } else {
            src = reinterpret_cast<const char*>(phiu + (long long)(tid - 9) * S + c);
            bytes = (unsigned)(w * sizeof(float));
        }
        const uintptr_t a = reinterpret_cast<uintptr_t>(src);
        const uintptr_t lo = (a + 15u) & ~uintptr_t(15), hi = (a + bytes) & ~uintptr_t(15);
        if (hi > lo)
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lo), "r"((unsigned)(hi - lo))
                         : "memory");
    };
    // A (asynchronous). phi of row Lr from the pairs this thread copied itself.
    auto lead_row_async = [&](int Lr) {
        cp_async_wait_all();
        if (ghost(Lr)) { ghost_row(Lr); return; }
        if (q0) phi_from_slot(Lr, 2 + 2 * tid);
        if (q1) phi_from_slot(Lr, 2 + 2 * (tid + TX));
    };
    // p of the previous step, row M (mirror ghost at walls), same column pairs.
    auto p_row = [&](int M) {
        const float* src = p_in + base + (ghost(M) ? mirror(M) : rowg(M)) * nx;
        float* dst = qrow(M);
        if (q0) st_pair(dst + 2 + 2 * tid, ld_pair(src + qc0));
        if (q1) st_pair(dst + 2 + 2 * (tid + TX), ld_pair(src + qc1));
    };
    // 3x3 neighbourhoods of the pair at ring index j (cells j, j+1) from three rows
    auto nbr_pair = [&](const float* r0, const float* r1, const float* r2, int j, Nbr<F2>& n) {
        const float* rows[3] = {r0, r1, r2};
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
            const float2 a2 = *reinterpret_cast<const float2*>(rows[dy] + j - 2);
            const float2 b2 = *reinterpret_cast<const float2*>(rows[dy] + j);
            const float2 c2 = *reinterpret_cast<const float2*>(rows[dy] + j + 2);
            n.z[dy][0] = F2(a2.y, b2.x);
            n.z[dy][1] = F2(b2);
            n.z[dy][2] = F2(b2.y, c2.x);
        }
    };
    // 3x3 neighbourhood of the low parts of phi around the pair at ring index j
    // of row M, from the h_0 pair slots of rows M - 1, M, M + 1 (all three are in
    // the slot window when mu of M is formed; a ghost row beyond a wall is its
    // mirror, the row next to it)
    auto lo_nbr = [&](int M, int j, Nbr<F2>& n) {
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
            const int r = M - 1 + dy;
            const float2* s2 = hpairs(ghost(r) ? mirror(r) : r);
            const float4 a4 = *reinterpret_cast<const float4*>(&s2[j - 2]);   // cells j-2, j-1
            const float4 b4 = *reinterpret_cast<const float4*>(&s2[j]);       // cells j, j+1
            const float4 c4 = *reinterpret_cast<const float4*>(&s2[j + 2]);   // cells j+2, j+3
            n.z[dy][0] = F2(a4.w, b4.y);
            n.z[dy][1] = F2(b4.y, b4.w);
            n.z[dy][2] = F2(b4.w, c4.y);
        }
    };
    // B. mu of row M (Eq. 8 with the Laplacian of Eq. 30b), same column pairs.
    auto mu_row = [&](int M) {
        float* dst = mrow(M);
        if (ghost(M)) {
            const float* src = mrow(mirror(M));
            if (q0) st_pair(dst + 2 + 2 * tid, lds_pair(src + 2 + 2 * tid));
            if (q1) st_pair(dst + 2 + 2 * (tid + TX), lds_pair(src + 2 + 2 * (tid + TX)));
            return;
        }
        const float *r0 = prow(M - 1), *r1 = prow(M), *r2 = prow(M + 1);
        auto column = [&](int q) {
            const int j = 2 + 2 * q;
            Nbr<F2> n;
            nbr_pair(r0, r1, r2, j, n);
            if constexpr (F::comp) {   // compensated: phi = hi + lo
                Nbr<F2> nl;
                lo_nbr(M, j, nl);
                st_pair(dst + j, chem_pot2(C, n.z[1][1], nl.z[1][1], n.lap() + nl.lap()));
            } else {
                st_pair(dst + j, chem_pot(C, n.z[1][1], n.lap()));
            }
        };
        if (q0) column(tid);
        if (q1) column(tid + TX);
    };
    // C. collision and push-streaming of the pair in row Y.
    auto collide_row = [&](int Y, const F2 (&g)[9], F2 pu_x, F2 pu_y) {
        if (!act) return;
        const int rY = rowoff(Y);
        const int c = rY + X;
        Nbr<F2> nphi, nmu, np;
        nbr_pair(prow(Y - 1), prow(Y), prow(Y + 1), jX, nphi);
        nbr_pair(mrow(Y - 1), mrow(Y), mrow(Y + 1), jX, nmu);
        nbr_pair(qrow(Y - 1), qrow(Y), qrow(Y + 1), jX, np);
        const F2 phi = nphi.z[1][1], mu = nmu.z[1][1];
        F2 gphix, gphiy, gmux, gmuy, gpx, gpy;
        nphi.grad(gphix, gphiy);
        nmu.grad(gmux, gmuy);
        np.grad(gpx, gpy);
        const F2 lapmu = nmu.lap();
        F2 h[9];
        F2 lo = F2(0.f);
        if constexpr (F::cons) {
            const float4 l4 = *reinterpret_cast<const float4*>(&hpairs(Y)[jX]);
            lo = F2(l4.y, l4.w);
            h[0] = lo;   // (not stored: the conservative h_0 is formed after the collision)
        }
#pragma unroll
        for (int i = F::cons ? 1 : 0; i < 9; ++i) h[i] = ld_pair(hplane(Y, i) + jX);   // as stored

        const Macro<F2> m = macroscopic<F::g16>(C, g, phi, mu, gphix, gphiy, gmux, gmuy, lapmu, gpx, gpy);
        const F2 phiux = phi * m.ux, phiuy = phi * m.uy;
        if constexpr (MON) {
            mon.add(phi, lo, m.rho, m.ux, m.uy);
        }
        // Push-streaming as each result is formed (halfway bounce-back into walls;
        // wall rows uniform per row). Conservative forms: h_0 goes last, as phi
        // minus the stored h_1..h_8 (per cell, as in step_kernel).
        const bool bot = walls && Y == 0, top = walls && Y == ny - 1;
        const int rDn = bot ? 0 : rowoff(Y - 1);
        const int rUp = top ? 0 : rowoff(Y + 1);
        // sums of the stored h_1..h_8 of the two cells (FP16 h: in units of hs)
        float ra = 0.f, rb = 0.f;
        collide_emit<F::g16, F::h16>(C, m, phi, mu, phiux - pu_x, phiuy - pu_y, g, h, [&](int i, F2 gi, F2 hi) {
            const auto gq = to_store(gi, gout);
            if constexpr (F::cons) {
                if (i == 0) {          // rest direction: g_0 now, h_0 after all h_1..h_8
                    st_both(gplane_out(0) + c, gq);
                    return;
                }
            }
            const auto hq = to_store(hi, hout);
            if constexpr (F::cons) {
                ra += first_f(hq);
                rb += second_f(hq);
            }
            const int cyi = cy_of(i), cxi = cx_of(i);
            if ((cyi > 0 && top) || (cyi < 0 && bot)) {   // back into the own pair, reversed
                const int k = opp_of(i);
                st_both(hplane_out(k) + c, hq);
                st_both(gplane_out(k) + c, gq);
                return;
            }
            const int r = cyi == 0 ? rY : (cyi > 0 ? rUp : rDn);
            if (cxi == 0) {
                if (!F::cons || i != 0) st_both(hplane_out(i) + r + X, hq);
                st_both(gplane_out(i) + r + X, gq);
            } else {
                const int da = r + (cxi > 0 ? X + 1 : colm);   // destination of cell X
                const int db = r + (cxi > 0 ? colp : X);       // destination of cell X + 1
                st_first(hplane_out(i) + da, hq);
                st_second(hplane_out(i) + db, hq);
                st_first(gplane_out(i) + da, gq);
                st_second(gplane_out(i) + db, gq);
            }
        });
        if constexpr (F::h16) {   // exact: ihs is a power of two
            ra *= ihs;
            rb *= ihs;
        }
        if constexpr (F::cons) {
            float s_, e_, hi, l2;
            float4 h0c;
            two_sum(phi.v.x, -ra, s_, e_);
            fast_two_sum(s_, e_ + lo.v.x, hi, l2);
            h0c.x = hi; h0c.y = l2;
            two_sum(phi.v.y, -rb, s_, e_);
            fast_two_sum(s_, e_ + lo.v.y, hi, l2);
            h0c.z = hi; h0c.w = l2;
            *reinterpret_cast<float4*>(h0out + c) = h0c;
        }
        st_pair(phiu + c, phiux);
        st_pair(phiu + S + c, phiuy);
        st_pair(p_out + c, m.p);
    };

    const int Y0 = wk.ystart;
    for (int pass = 0; pass < 2; ++pass)
        for (int k = 1; k >= -2; --k)
            if (ghost(Y0 + k * d) == (pass == 1)) lead_row(Y0 + k * d);
    p_row(Y0 - d);
    p_row(Y0);
    group_sync(bar, TX);
    mu_row(Y0);
    mu_row(Y0 - d);
    if constexpr (F::comp) {
        // mu of row Y0 - d read the low parts of phi from the h slot of row
        // Y0 - 2d: every thread must be done with it before it is refilled
        group_sync(bar, TX);
        prefetch(Y0 + 2 * d, Y0 + d);   // the slot of row Y0 - 2d takes the first lead row
    } else {
        // (issued before the barrier: the slot of row Y0 - 2d was read only above)
        prefetch(Y0 + 2 * d, Y0 + d);
        group_sync(bar, TX);
    }
    for (int k = 0; k < wk.nrows; ++k) {
        const int Y = Y0 + k * d;
        // g and phi*u of the collision pair, loaded before the barriers
        F2 g[9];
        F2 pux = F2(0.f), puy = F2(0.f);
        if (act) {
            const int c = rowoff(Y) + X;
#pragma unroll
            for (int i = 0; i < 9; ++i) g[i] = ld_g(i, c);
            pux = ld_pair(phiu + c);
            puy = ld_pair(phiu + S + c);
        }
        // the next collision row's g and phi*u into L2, issued with this row's loads
        // (measured on the 1024 x 4096 bubble, FP32 h: +11 % against no prefetch;
        // later in the iteration or further ahead gained less, lost from three
        // rows ahead; FP16 h: no gain)
        if constexpr (!F::h16)
            if (k + 1 < wk.nrows) l2_prefetch_row(Y + d);
        lead_row_async(Y + 2 * d);
        group_sync(bar, TX);
        // every thread is past the collision of row Y - d: the h slot of row Y - d
        // and the p slot of row Y - 2d are free for the next iteration's rows
        if (k + 1 < wk.nrows) prefetch(Y + 3 * d, Y + 2 * d);
        mu_row(Y + d);
        group_sync(bar, TX);
        collide_row(Y, g, pux, puy);
    }
    if constexpr (MON == 1) mon_block_store(mon, a, wk.inst, item, wk.pad, tid, TX, bar, grp);
    if constexpr (MON == 2) {
        // persistent launch: publish this item's step first (the monitor's tree
        // reads only the monitor buffers), so the neighbour items' next step
        // need not wait for the reduction
        group_sync(bar, TX);
        if (tid == 0) {
            __threadfence();
            atomicAdd(a.done + item, 1);
        }
        mon_step_store(mon, a, wk.inst, item, wk.pad, tid, TX, bar, grp, step);
    }
}

template <int FORM, int TX, bool MON = false>
__global__ void __launch_bounds__(TX, X2Occ<FORM, TX>::value) step_kernel_x2(const StepArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    x2_item<FORM, MON>(a, blockIdx.x, smem_raw, threadIdx.x, 0, 0, TX);
}

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// ---------------------------------------------------------------------------
// Several steps of one plan of work items in one persistent launch (the
// LBM_PIPELINE_PERSISTENT plan of a context whose items all fit on the GPU at
// once): block b owns work item b for every step, and before step s > 0 waits
// only until each of its neighbour items (a.nbr[b * kMaxNbr ..], -1 padded:
// the items whose rows and columns lie within the 3 rows and 2 columns one step
// reads or writes around item b) has finished step s - 1, counted in a.done
// (zeroed before the launch). Those are exactly the items that read what step
// s of b overwrites and wrote what it reads, so no grid-wide step boundary is
// needed; neighbours stay within one step of each other. The launch is
// cooperative (every block resident), so every wait ends; each is bounded all
// the same (a.wait_limit rounds): one that runs out records a timeout in the
// status word, raises the abort flag a.done[a.ndesc] and the block leaves, as
// do the blocks waiting on it. Odd steps read the other buffer set (swap).
// MON: every step's monitor record as well (mon_step_store).
template <int FORM, int TX, bool MON = false>
__global__ void __launch_bounds__(TX, X2Occ<FORM, TX>::value) step_kernel_x2_multi(const StepArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_bad;
    const int b = blockIdx.x, tid = threadIdx.x;
    int* abort_flag = a.done + a.ndesc;
    for (int s = 0; s < a.nsteps; ++s) {
        if (s > 0) {
            if (tid < 32) {
                int ok = 1;
                if (tid < kMaxNbr) {
                    const int n = a.nbr[b * kMaxNbr + tid];
                    if (n >= 0) {
                        const int need = s + a.wait_extra;
                        ok = 0;
                        for (int it = 0; it < a.wait_limit; ++it) {
                            if (ld_acquire_gpu(a.done + n) >= need) {
                                ok = 1;
                                break;
                            }
                            if (*reinterpret_cast<volatile int*>(abort_flag)) break;
                            __nanosleep(64);
                        }
                        __threadfence();
                    }
                }
                const unsigned bad = __ballot_sync(0xffffffffu, !ok);
                if (tid == 0) {
                    if (bad) {
                        atomicExch(a.status, kStatusTimeout);
                        atomicExch(abort_flag, 1);
                    }
                    s_bad = bad != 0;
                }
            }
            __syncthreads();
            if (s_bad) return;
        }
        x2_item<FORM, MON ? 2 : 0>(a, b, smem_raw, tid, 0, 0, TX, (s & 1) != 0, s);
        __syncthreads();   // every thread's stores of step s issued
        if (!MON && tid == 0) {   // (the monitored item publishes itself, before its monitor tree)
            __threadfence();
            atomicAdd(a.done + b, 1);
        }
    }
}

// ---------------------------------------------------------------------------
// The batched step: every instance of a context, several steps, in one
// persistent launch. Blocks of 128 threads take (step, block descriptor) pairs
// from a queue -- an atomic counter over nsteps x ndesc, step-major; within a
// step the planner sorts the descriptors longest run first -- until it runs
// dry. A descriptor holds either one wide item (a strip of up to 256 columns,
// marched by all 128 threads; item[1] == kDescWide) or two narrow ones (strips
// of up to 128 columns, each on its own group of 64 threads with its own
// shared-memory region and named barrier, so the two groups march
// independently: different instances, run lengths and directions). Both kinds
// go through one inlined x2_item with the group width as a run-time value (two
// inlined bodies, one a width, made the register allocator spill).
// Steps overlap across instances: an item of step s > 0 waits only until every
// item of its own instance's step s - 1 has finished (a per-instance counter of
// finished items), so no grid-wide step boundary leaves SMs idle in a tail. The
// wait is safe: items are handed out in step order, so every item waited for
// was taken earlier by a running block, and the earliest unfinished one waits
// for nothing. It is bounded all the same: after wait_limit rounds the group
// records a timeout in the status word, raises the abort flag (every block
// then stops taking work) and skips its item. The last block to finish sets
// the queue and the counters back to zero for the next launch.
// Three resident blocks a SM (up to 168 registers a thread) for every form: at
// four, the FP16-h form's batched kernel spilled at its 128-register cap and ran
// at 23.2k MLUPS on the 512 mixed instances.
template <int FORM>
struct X2Batched {
    static constexpr size_t narrow = X2Smem<FORM, 64>::bytes;    // one group of 64
    static constexpr size_t wide = X2Smem<FORM, 128>::bytes;     // the block as one group
    static constexpr size_t bytes = 2 * narrow > wide ? 2 * narrow : wide;
    static constexpr int by_smem = (int)((228u * 1024u) / (bytes + 1024u));
    static constexpr int occ = by_smem < 3 ? by_smem : 3;
};

template <int FORM, bool MON = false>
__global__ void __launch_bounds__(128, X2Batched<FORM>::occ) step_kernel_x2_batched(const StepArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_desc, s_abort;
    __shared__ int s_skip[2];
    const int tid = threadIdx.x;
    const int g = tid >> 6;   // narrow thread group: 0 or 1
    const int total = a.nsteps * a.ndesc;
    volatile int* abort_flag = a.queue + 2;
    for (;;) {
        if (tid == 0) {
            s_desc = atomicAdd(a.queue, 1);
            s_abort = *abort_flag;
        }
        __syncthreads();
        const int gq = s_desc;
        if (gq >= total || s_abort) break;
        const int s = gq / a.ndesc, q = gq - s * a.ndesc;
        const int i0 = a.desc[q].item[0], i1 = a.desc[q].item[1];
        const bool wide = i1 == kDescWide;
        const int item = (wide || g == 0) ? i0 : i1;
        const int gt = wide ? tid : tid & 63, nthr = wide ? 128 : 64, bar = wide ? 1 : 1 + g, grp = wide ? 0 : g;
        int inst = -1;
        bool run = item >= 0;
        if (run) {
            inst = a.work[item].inst;
            if (s > 0) {   // every item of this instance's step s - 1 finished
                if (gt == 0) {
                    const int need = s * (a.items_csr[inst + 1] - a.items_csr[inst]) + a.wait_extra;
                    int ok = 0;
                    for (int it = 0; it < a.wait_limit; ++it) {
                        if (ld_acquire_gpu(a.done + inst) >= need) {
                            ok = 1;
                            break;
                        }
                        if (*abort_flag) break;
                        __nanosleep(64);
                    }
                    if (!ok) {
                        atomicExch(a.status, kStatusTimeout);
                        atomicExch(a.queue + 2, 1);
                    }
                    __threadfence();
                    s_skip[grp] = !ok;
                }
                group_sync(bar, nthr);
                run = !s_skip[grp];
            }
            if (run)
                x2_item<FORM, MON>(a, item, smem_raw + (wide ? 0 : g * X2Batched<FORM>::narrow), gt, bar, grp,
                                   nthr, !MON && (s & 1) != 0);   // a monitored launch runs one step
        }
        __syncthreads();   // the groups are done with their regions and stores; s_desc may change
        if (run && gt == 0) {   // publish: one more item of this instance finished
            __threadfence();
            atomicAdd(a.done + inst, 1);
        }
    }
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(a.queue + 1, 1) == (int)gridDim.x - 1) {   // every block is past the queue
            for (int k = 0; k < a.ninst; ++k) a.done[k] = 0;
            a.queue[0] = 0;
            a.queue[1] = 0;
            a.queue[2] = 0;
            __threadfence();
        }
    }
}

}  // namespace lbm
