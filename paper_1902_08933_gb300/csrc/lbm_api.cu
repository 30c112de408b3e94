// lbm_api.cu -- the C ABI of include/lbm.h: contexts, device memory, work
// planning, kernel dispatch, field readback, diagnostics and checkpoints.
#include <algorithm>
#include <cstddef>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_internal.h"
#include "lbm_mbar.cuh"

using lbm::AuxArgs;
using lbm::DevInst;
using lbm::StepArgs;
using lbm::WorkItem;

namespace {

constexpr int kForms = 6;

template <typename Fn>
cudaError_t by_form(int form, Fn&& fn) {
    switch (form) {
        case 0: return fn(std::integral_constant<int, 0>{});
        case 1: return fn(std::integral_constant<int, 1>{});
        case 2: return fn(std::integral_constant<int, 2>{});
        case 3: return fn(std::integral_constant<int, 3>{});
        case 4: return fn(std::integral_constant<int, 4>{});
        case 5: return fn(std::integral_constant<int, 5>{});
        default: return cudaErrorInvalidValue;
    }
}

// storage of each form (see the form table in lbm_device.cuh)
size_t h_elem(int form) { return form == 0 ? 8 : (form == 3 ? 2 : 4); }
size_t g_elem(int form) { return form == 0 ? 8 : ((form == 2 || form == 3) ? 2 : 4); }
size_t a_elem(int form) { return form == 0 ? 8 : 4; }
bool conservative(int form) { return form >= 2; }
int h_planes(int form, int q = 9) { return conservative(form) ? q - 1 : q; }
// lattice of an instance: nz >= 2 selects D3Q15 (Sec. 2.2)
bool is_d3(const lbm_params& p) { return p.nz >= 2; }
long long cells_of(const lbm_params& p) { return (long long)p.nx * p.ny * (is_d3(p) ? p.nz : 1); }

// Largest power of two s with s * bound <= 2048: keeps FP16-stored values
// (|v| * s) at least 30x below the FP16 maximum and far above its subnormals.
double pow2_scale(double bound) {
    if (!(bound > 0)) return 1.0;
    return std::ldexp(1.0, (int)std::floor(std::log2(2048.0 / bound)));
}

bool finite_all(const lbm_params& p) {
    const double v[] = {p.rho_A, p.rho_B, p.nu_A, p.nu_B, p.sigma, p.W, p.tau_h,
                        p.mobility, p.force_x, p.force_y, p.gravity};
    for (double x : v)
        if (!std::isfinite(x)) return false;
    return true;
}

const char* check_params(const lbm_params& p) {
    if (p.nx < 3 || p.ny < 3) return "nx and ny must be >= 3";
    if (p.nz < 0) return "nz must be >= 0";
    if (cells_of(p) >= (1LL << 31)) return "nx*ny*nz must be < 2^31";
    if (p.bc_y != LBM_BC_PERIODIC && p.bc_y != LBM_BC_BOUNCEBACK) return "bc_y out of range";
    if (p.variant != LBM_IM && p.variant != LBM_QIM) return "variant out of range";
    if (p.pressure_scheme < LBM_P_MODIFIED_PRINTED || p.pressure_scheme > LBM_P_PREVIOUS)
        return "pressure_scheme out of range";
    if (p.surface_force != LBM_FS_MU_GRADPHI && p.surface_force != LBM_FS_PHI_GRADMU)
        return "surface_force out of range";
    if (p.viscosity_model != LBM_VISC_INV_LINEAR && p.viscosity_model != LBM_VISC_STEP)
        return "viscosity_model out of range";
    if (!finite_all(p)) return "parameters must be finite";
    if (!(p.rho_A > 0 && p.rho_B > 0)) return "densities must be > 0";
    if (!(p.nu_A > 0 && p.nu_B > 0)) return "viscosities must be > 0";
    if (!(p.W > 0)) return "W must be > 0";
    if (!(p.sigma >= 0)) return "sigma must be >= 0";
    if (!(p.mobility >= 0)) return "mobility must be >= 0";
    if (!(p.tau_h > 0.5)) return "tau_h must be > 1/2";
    return nullptr;
}

// Host-side derivation of the per-instance constants (Eqs. 6-7, 17, Sec. 3.2.1).
DevInst derive(const lbm_params& p, long long base, int form) {
    DevInst d;
    std::memset(&d, 0, sizeof(d));
    d.base = base;
    d.nx = p.nx;
    d.ny = p.ny;
    d.nz = is_d3(p) ? p.nz : 1;
    d.walls = p.bc_y == LBM_BC_BOUNCEBACK;
    d.qim = p.variant == LBM_QIM;
    d.pscheme = p.pressure_scheme;
    d.sforce = p.surface_force;
    d.visc = p.viscosity_model;
    d.uniform_nu = (p.viscosity_model == LBM_VISC_INV_LINEAR && p.nu_A == p.nu_B) ? 1 : 0;
    d.tgm0 = 3.0 * p.nu_A;                         // nu = c_s^2 (tau_g - 1/2)
    d.inv_tau_g0 = 1.0 / (d.tgm0 + 0.5);
    const double phiA = 1.0, phiB = 0.0;
    d.rho_A = p.rho_A;
    d.rho_B = p.rho_B;
    d.drho = (p.rho_A - p.rho_B) / (phiA - phiB);
    d.inv_nu_A = 1.0 / p.nu_A;
    d.inv_nu_B = 1.0 / p.nu_B;
    d.mu_A = p.rho_A * p.nu_A;
    d.mu_B = p.rho_B * p.nu_B;
    d.kappa = 1.5 * p.sigma * p.W;                 // from W = sqrt(8 kappa / beta), sigma = sqrt(2 kappa beta)/6
    d.beta = 12.0 * p.sigma / p.W;
    d.eta = p.mobility / ((1.0 / 3.0) * (p.tau_h - 0.5));   // Eq. 17
    const double gamma = (p.rho_A - p.rho_B) / (phiA * p.rho_B - phiB * p.rho_A);
    d.gammaM = gamma * p.mobility;
    d.inv_tau_h = 1.0 / p.tau_h;
    d.force_x = p.force_x;
    d.force_y = p.force_y;
    d.gravity = p.gravity;
    // Storage scales of the FP16 forms: bounds of |h_i| (i != 0) and |g_i| from the
    // equilibria (Eqs. 11, 33) with |mu| <~ beta and |u| <~ 0.1.
    const double rho_max = std::max(p.rho_A, p.rho_B);
    const double h_bound = (d.eta * d.beta + 0.35) / 9.0;
    const double g_bound = rho_max * 0.05 + 3.0 * d.beta + 1e-3;
    d.h_scale = form == 3 ? pow2_scale(h_bound) : 1.0;
    d.g_scale = (form == 2 || form == 3) ? pow2_scale(g_bound) : 1.0;
    return d;
}

}  // namespace

struct lbm_ctx {
    int n = 0, form = 0, device = 0;
    bool d3 = false;                 // D3Q15 lattice (every instance)
    int q = 9;                       // populations a set: 9 (D2Q9) or 15 (D3Q15)
    lbm::D3Scratch sc{nullptr, nullptr, nullptr};   // D3Q15 scratch planes
    std::vector<lbm_params> params;
    std::vector<DevInst> inst;
    std::vector<int64_t> time;
    std::vector<char> ready;
    long long S = 0, max_cells = 0;
    DevInst* d_inst = nullptr;
    // The two buffer sets (time levels) of h, h_0, g and p, in one allocation:
    // set b at state + b * set_bytes, each array at the same offset in both, so
    // that one signed byte offset takes every array to the other set (what the
    // batched launch's odd steps add, see StepArgs::set_delta).
    void* state = nullptr;
    long long set_bytes = 0;
    void* h[2] = {nullptr, nullptr};
    void* h0[2] = {nullptr, nullptr};     // conservative forms: h_0 as float2
    void* g[2] = {nullptr, nullptr};
    void* phiu = nullptr;
    void* p[2] = {nullptr, nullptr};
    int cur = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int tile_req = 0, rows_req = 0;
    int pipeline = LBM_PIPELINE_AUTO;
    int* d_status = nullptr;       // device status word written by bounded waits
    struct Launch { int tx, offset, count, variant; };
    std::vector<Launch> launches;
    std::vector<WorkItem> work;
    WorkItem* d_work = nullptr;
    // batched step (one persistent launch over all instances): block descriptors
    // and the queue counters the kernel takes them with
    lbm::BlockDesc* d_desc = nullptr;
    int ndesc = 0;
    int* d_queue = nullptr;        // batched queue: next, blocks finished, abort
    int* d_done = nullptr;         // batched: items finished a launch, per instance
    bool multi = false;            // persistent plan: several steps a launch
    long long step_launches = 0;   // kernel launches lbm_step has issued (graph nodes counted)
    int graph_launches = 0;        // kernel nodes of the captured graph
    int* d_nbr = nullptr;          // persistent plan: neighbour items, kMaxNbr an item
    int* d_multi_done = nullptr;   // persistent plan: steps finished per item, then the abort flag
    double* d_mon_multi = nullptr; // persistent plan, every step monitored: [64 steps][items][kMonQ] slots
    int* d_mon_multi_cnt = nullptr;   // ... [64 steps][instances][kMonSub + 1] counters
    double* d_mon_multi_sub = nullptr;  // ... and [64 steps][instances][kMonSub][kMonQ] sub-group slots
    bool plan_dirty = true;
    // CUDA graph of 2 * graph_pairs steps starting from cur == 0 (built on first use,
    // dropped when the plan changes)
    cudaGraphExec_t graph = nullptr;
    int graph_steps = 0;
    // graph capture with several launch classes: one branch per class
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    // per-step monitor of the last step of each lbm_step call
    bool monitor = false;
    double* d_mon_partials = nullptr;   // kMonQ doubles per work item
    int* d_mon_csr = nullptr;           // per instance: work items [ptr[k], ptr[k+1]) of idx
    int* d_mon_count = nullptr;         // per instance: the reduction tree's counters (0 between steps)
    double* d_mon_sub = nullptr;        // per instance: kMonSub sub-group slots
    lbm_monitor* d_mon = nullptr;       // one record per instance
    lbm::MonRecord* mon_host_dev = nullptr;   // during lbm_step_monitored: the caller's mapped host records
    int64_t steps_total = 0;            // steps taken by the context
    int64_t* d_time_base = nullptr;     // per instance: time - steps_total (device copy)
    lbm_monitor* h_mon = nullptr;       // pinned staging record
    std::vector<int64_t> mon_time;      // time level of the recorded sums (-1: none)
    bool use_graphs = true;
    double* d_tmp = nullptr;       // 2 * max_cells
    double* d_out = nullptr;       // field staging, grown on demand
    size_t d_out_cells = 0;
    double* d_partials = nullptr;
    double* d_result = nullptr;
    double* h_result = nullptr;    // pinned
    std::string err;
};

namespace {

lbm_status fail(lbm_ctx* c, lbm_status st, const std::string& msg) {
    if (c) c->err = msg;
    return st;
}

lbm_status cuda_fail(lbm_ctx* c, cudaError_t e, const char* what) {
    return fail(c, LBM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define LBM_CK(ctx, call)                                          \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call); \
    } while (0)

StepArgs step_args(const lbm_ctx* c, int in) {
    StepArgs a;
    a.h_in = c->h[in];
    a.h_out = c->h[1 - in];
    a.h0_in = c->h0[in];
    a.h0_out = c->h0[1 - in];
    a.g_in = c->g[in];
    a.g_out = c->g[1 - in];
    a.phiu = c->phiu;
    a.p_in = c->p[in];
    a.p_out = c->p[1 - in];
    a.set_delta = in == 0 ? c->set_bytes : -c->set_bytes;
    a.S = c->S;
    a.inst = c->d_inst;
    a.work = nullptr;
    a.status = c->d_status;
    a.mon = nullptr;
    a.mon_all = nullptr;
    a.mon_sub = nullptr;
    a.mon_count = nullptr;
    a.mon_csr = nullptr;
    a.mon_n = 0;
    a.mon_rec = nullptr;
    a.time_base = nullptr;
    a.mon_step = 0;
    a.desc = c->d_desc;
    a.ndesc = c->ndesc;
    a.queue = c->d_queue;
    a.done = c->d_done;
    a.items_csr = c->d_mon_csr;
    a.nbr = nullptr;
    a.ninst = c->n;
    a.nsteps = 1;
    a.wait_limit = lbm::kWaitLimit;
    a.wait_extra = 0;
    a.mon_host = nullptr;
    return a;
}

AuxArgs aux_args(const lbm_ctx* c, int instance) {
    AuxArgs a;
    std::memset(&a, 0, sizeof(a));
    a.h = c->h[c->cur];
    a.h0 = c->h0[c->cur];
    a.g = c->g[c->cur];
    a.phiu = c->phiu;
    a.p_prev = c->p[c->cur];
    a.S = c->S;
    a.inst = c->d_inst;
    a.instance = instance;
    a.tmp_phi = c->d_tmp;
    a.tmp_mu = c->d_tmp + c->max_cells;
    a.partials = c->d_partials;
    a.result = c->d_result;
    return a;
}

int default_tile(int nx) {
    if (nx >= 128) return 128;
    if (nx > 32) return 64;
    return 32;
}

int default_tile_pairs(int nx) {   // strip width of the paired kernel (2 columns a thread)
    if (nx >= 256) return 256;
    if (nx >= 128) return 128;
    return 64;
}

// Load path and strip width of one instance under the context's pipeline mode.
// The paired kernel needs nx even and strips of at least 64 columns; the TMA-fed
// kernel 16-byte row segments (nx % 8 == 0, see lbm_step_tma.cuh); both exist for
// the FP32-arithmetic forms, the cp.async kernel for FP32 storage of h and p.
void choose(const lbm_ctx* c, const lbm_params& p, bool f_pairs, bool f_async, bool f_tma,
            int* tile, int* variant, int mode = -1) {
    const bool pairs_ok = f_pairs && p.nx % 2 == 0 && (c->tile_req == 0 || c->tile_req >= 64);
    const bool tma_ok = f_tma && p.nx % 8 == 0 && p.nx >= 8;
    int v = lbm::kPlain;
    switch (mode < 0 ? c->pipeline : mode) {
        case LBM_PIPELINE_AUTO:
        case LBM_PIPELINE_BATCHED:   // (when the batched launch does not apply)
            v = pairs_ok ? lbm::kPairs : (f_async ? lbm::kAsync : (tma_ok ? lbm::kTma : lbm::kPlain));
            break;
        case LBM_PIPELINE_PAIRS:
        case LBM_PIPELINE_PERSISTENT: v = pairs_ok ? lbm::kPairs : lbm::kPlain; break;
        case LBM_PIPELINE_ASYNC: v = f_async ? lbm::kAsync : lbm::kPlain; break;
        case LBM_PIPELINE_TMA: v = tma_ok ? lbm::kTma : lbm::kPlain; break;
        default: v = lbm::kPlain; break;
    }
    *variant = v;
    if (c->tile_req) *tile = c->tile_req;
    else *tile = v == lbm::kPairs ? default_tile_pairs(p.nx) : default_tile(p.nx);
}

// Work list: per instance, strips of tile_x columns, each split into runs of
// rows, grouped into one launch per (strip width, load path). Neighbouring runs
// march in opposite directions (down, up, down, ...) so that two blocks that
// share a run boundary read its halo rows at the same time (both at their start
// or both at their end), from L2 rather than HBM.
lbm_status plan_d3(lbm_ctx* c);
lbm_status plan_multi(lbm_ctx* c, int sms);
lbm_status plan_batched(lbm_ctx* c, bool f_pairs, bool f_async, bool f_tma, int sms);
lbm_status finish_plan(lbm_ctx* c);

// The batched launch serves a context when asked for (LBM_PIPELINE_BATCHED) or,
// under LBM_PIPELINE_AUTO, when it holds several instances; in both cases only
// if every instance can use the paired kernel.
bool use_batched(const lbm_ctx* c, bool f_pairs, bool f_async, bool f_tma) {
    if (c->d3 || !f_pairs) return false;
    if (c->pipeline != LBM_PIPELINE_BATCHED && !(c->pipeline == LBM_PIPELINE_AUTO && c->n > 1)) return false;
    for (const lbm_params& p : c->params) {
        int tx = 0, variant = 0;
        choose(c, p, f_pairs, f_async, f_tma, &tx, &variant, LBM_PIPELINE_PAIRS);
        if (variant != lbm::kPairs) return false;
    }
    return true;
}

lbm_status plan(lbm_ctx* c) {
    if (c->d3) return plan_d3(c);
    const int tiles[4] = {32, 64, 128, 256};
    auto tile_index = [&](int tx) {
        for (int k = 0; k < 4; ++k)
            if (tiles[k] == tx) return k;
        return 0;
    };
    std::vector<std::vector<WorkItem>> by_class(16);   // tile index * 4 + variant
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    bool f_pairs = false, f_async = false, f_tma = false;
    by_form(c->form, [&](auto F) {
        f_pairs = lbm::has_pairs_t<decltype(F)::value>();
        f_async = lbm::has_async_t<decltype(F)::value>();
        f_tma = lbm::has_tma_t<decltype(F)::value>();
        return cudaSuccess;
    });
    if (use_batched(c, f_pairs, f_async, f_tma)) return plan_batched(c, f_pairs, f_async, f_tma, sms);
    // Several instances: one run length for all, sized for about four waves of
    // blocks (blocks of different instances differ in width and length, so one
    // exact wave cannot be had; shorter runs balance better but re-read more
    // halo rows -- 4 a run, mostly from L2 -- and the launch classes overlap as
    // graph branches, which takes up much of the imbalance). Tiny batches get
    // 1-row runs: there the step is bound by the latency of a block's row march.
    int batch_rows = 32;
    if (c->n > 1) {
        long long strip_rows = 0;
        int occ_min = 1 << 30;
        for (int k = 0; k < c->n; ++k) {
            int tx = 0, variant = 0;
            choose(c, c->params[k], f_pairs, f_async, f_tma, &tx, &variant);
            strip_rows += (long long)((c->params[k].nx + tx - 1) / tx) * c->params[k].ny;
            int occ = 0;
            by_form(c->form, [&](auto F) {
                occ = lbm::step_occupancy_t<decltype(F)::value>(tx, variant);
                return cudaSuccess;
            });
            occ_min = std::min(occ_min, std::max(occ, 1));
        }
        const long long target = 4LL * sms * occ_min;
        batch_rows = (int)std::max<long long>(1, std::min<long long>(64, strip_rows / target));
    }
    for (int k = 0; k < c->n; ++k) {
        const lbm_params& p = c->params[k];
        int tx = 0, variant = 0;
        choose(c, p, f_pairs, f_async, f_tma, &tx, &variant);
        const int strips = (p.nx + tx - 1) / tx;
        int rows = c->rows_req;
        if (rows <= 0) {
            if (c->n == 1) {
                // one domain: fill the GPU with resident blocks in a single wave
                int occ = 0;
                by_form(c->form, [&](auto F) {
                    occ = lbm::step_occupancy_t<decltype(F)::value>(tx, variant);
                    return cudaSuccess;
                });
                // runs per strip: least (waves) x (rows a run + 3 for the prologue),
                // waves counted whole -- one exact wave where the strips allow it
                const long long target = (long long)sms * std::max(occ, 1);
                long long best = -1, best_cost = 0;
                for (long long r = 1; r <= p.ny; ++r) {
                    const long long rr = (p.ny + r - 1) / r;
                    if (rr < 8 && r > 1) break;   // runs of at least 8 rows
                    const long long runs = (p.ny + rr - 1) / rr;
                    const long long waves = (strips * runs + target - 1) / target;
                    const long long cost = waves * (rr + 3);
                    if (best < 0 || cost < best_cost) { best = rr; best_cost = cost; }
                }
                rows = (int)best;
            } else {
                rows = batch_rows;
            }
        }
        rows = std::min(rows, p.ny);
        const int nchunks = (p.ny + rows - 1) / rows;
        auto& list = by_class[tile_index(tx) * 4 + variant];
        for (int s = 0; s < strips; ++s)
            for (int ch = 0; ch < nchunks; ++ch) {
                const int y0 = ch * rows, y1 = std::min(p.ny, y0 + rows);
                WorkItem w;
                w.inst = k;
                w.x0 = s * tx;
                w.nrows = y1 - y0;
                w.dir = (ch % 2 == 0) ? -1 : 1;
                w.ystart = w.dir < 0 ? y1 - 1 : y0;
                w.pad = 0;
                list.push_back(w);
            }
    }
    c->work.clear();
    c->launches.clear();
    for (int k = 0; k < 16; ++k) {
        if (by_class[k].empty()) continue;
        c->launches.push_back({tiles[k / 4], (int)c->work.size(), (int)by_class[k].size(), k % 4});
        c->work.insert(c->work.end(), by_class[k].begin(), by_class[k].end());
    }
    c->ndesc = 0;
    lbm_status st = finish_plan(c);
    if (st != LBM_OK) return st;
    return plan_multi(c, sms);
}

// Batched plan: the paired kernel's work items of every instance, runs of rows
// with alternating directions. Instances wider than 128 columns are cut into
// strips of 256 (wide items: one a block descriptor, all 128 threads on it --
// the strip width of the one-instance launch, measured 12 % faster than 128 on
// the 512 mixed instances); narrower instances, and a last strip of at most 128
// columns, are narrow items, paired into descriptors (items of equal run length
// together). The descriptors are sorted by run length, longest first, so the
// queue hands out the long ones first and the short ones fill the tail. Run
// length: about one descriptor per resident block a step, at most 64 rows,
// unless set by lbm_set_launch (its strip width does not apply here) -- long
// runs re-read fewer halo rows, and the tail of a step is hidden by the next
// step's items of the instances already done (several steps a launch): on the
// 512 mixed instances 64-row runs beat 32 by 4 % (FP32) and 16 by 12 %.
lbm_status plan_batched(lbm_ctx* c, bool, bool, bool, int sms) {
    int occ = 1;
    by_form(c->form, [&](auto F) {
        occ = std::max(1, lbm::batched_occupancy_t<decltype(F)::value>());
        return cudaSuccess;
    });
    constexpr int kWideStrip = 256, kNarrowStrip = 128;
    // strips of one instance: (x0, width) with width > kNarrowStrip for wide ones
    auto strips_of = [&](const lbm_params& p) {
        std::vector<std::pair<int, int>> v;
        for (int x0 = 0; x0 < p.nx;) {
            const int w = p.nx - x0 > kNarrowStrip ? std::min(kWideStrip, p.nx - x0) : p.nx - x0;
            v.push_back({x0, w});
            x0 += w;
        }
        return v;
    };
    int rows = c->rows_req;
    if (rows <= 0) {
        double block_rows = 0;   // rows of whole blocks: a narrow item is half a block
        for (const lbm_params& p : c->params)
            for (const auto& sw : strips_of(p)) block_rows += (sw.second > kNarrowStrip ? 1.0 : 0.5) * p.ny;
        rows = (int)std::lround(block_rows / (1.0 * sms * occ));
        rows = std::max(8, std::min(64, rows));
    }
    std::vector<WorkItem> wide, narrow;
    for (int k = 0; k < c->n; ++k) {
        const lbm_params& p = c->params[k];
        const int r = std::min(rows, p.ny);
        const int nchunks = (p.ny + r - 1) / r;
        for (const auto& sw : strips_of(p))
            for (int ch = 0; ch < nchunks; ++ch) {
                const int y0 = ch * r, y1 = std::min(p.ny, y0 + r);
                WorkItem w;
                w.inst = k;
                w.x0 = sw.first;
                w.nrows = y1 - y0;
                w.dir = (ch % 2 == 0) ? -1 : 1;
                w.ystart = w.dir < 0 ? y1 - 1 : y0;
                w.pad = 0;
                (sw.second > kNarrowStrip ? wide : narrow).push_back(w);
            }
    }
    auto longer = [](const WorkItem& x, const WorkItem& y) { return x.nrows > y.nrows; };
    std::stable_sort(narrow.begin(), narrow.end(), longer);
    c->work = wide;
    c->work.insert(c->work.end(), narrow.begin(), narrow.end());
    std::vector<lbm::BlockDesc> host;
    std::vector<int> len;
    for (int j = 0; j < (int)wide.size(); ++j) {
        host.push_back({{j, lbm::kDescWide}});
        len.push_back(wide[j].nrows);
    }
    const int nw = (int)wide.size(), nn = (int)narrow.size();
    for (int j = 0; j < nn; j += 2) {
        host.push_back({{nw + j, j + 1 < nn ? nw + j + 1 : -1}});
        len.push_back(narrow[j].nrows);   // the longer of the two
    }
    std::vector<int> order(host.size());
    for (int i = 0; i < (int)order.size(); ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return len[x] > len[y]; });
    {
        std::vector<lbm::BlockDesc> sorted;
        for (int i : order) sorted.push_back(host[i]);
        host.swap(sorted);
    }
    c->ndesc = (int)host.size();
    c->launches.clear();
    c->launches.push_back({kNarrowStrip, 0, (int)std::min<long long>(c->ndesc, (long long)sms * occ), lbm::kBatched});
    cudaFree(c->d_desc);
    c->d_desc = nullptr;
    LBM_CK(c, cudaMalloc(&c->d_desc, host.size() * sizeof(lbm::BlockDesc)));
    LBM_CK(c, cudaMemcpy(c->d_desc, host.data(), host.size() * sizeof(lbm::BlockDesc), cudaMemcpyHostToDevice));
    if (!c->d_queue) LBM_CK(c, cudaMalloc(&c->d_queue, 4 * sizeof(int)));
    LBM_CK(c, cudaMemset(c->d_queue, 0, 4 * sizeof(int)));
    if (!c->d_done) LBM_CK(c, cudaMalloc(&c->d_done, (size_t)c->n * sizeof(int)));
    LBM_CK(c, cudaMemset(c->d_done, 0, (size_t)c->n * sizeof(int)));
    return finish_plan(c);
}

// The persistent plan (LBM_PIPELINE_PERSISTENT): a paired plan of one launch
// class whose blocks all fit on the GPU at once runs several steps a launch
// (step_kernel_x2_multi). Neighbour lists: for each item, the other items of its
// instance whose columns lie within 2 and whose rows lie within 3 of its own
// (periodic where the instance is; the reach of one step of the row march: lead
// rows 2 ahead, pushes 1 row and 1 column out, the phi halo 2 columns). More
// than kMaxNbr neighbours, or more items than resident blocks: no persistent
// launch, the plan runs as PAIRS.
// steps of one monitored persistent launch (slots and counters are kept per step)
constexpr int kMultiSteps = 64;

lbm_status plan_multi(lbm_ctx* c, int sms) {
    c->multi = false;
    if (c->d3 || c->pipeline != LBM_PIPELINE_PERSISTENT || c->launches.size() != 1 ||
        c->launches[0].variant != lbm::kPairs)
        return LBM_OK;
    const auto& L = c->launches[0];
    int occ = 0;
    by_form(c->form, [&](auto F) {
        occ = lbm::multi_occupancy_t<decltype(F)::value>(L.tx);
        return cudaSuccess;
    });
    if (occ <= 0 || (long long)L.count > (long long)sms * occ) return LBM_OK;
    struct Box { int inst, x0, x1, y0, y1; };
    std::vector<Box> box(L.count);
    for (int k = 0; k < L.count; ++k) {
        const WorkItem& w = c->work[L.offset + k];
        const lbm_params& p = c->params[w.inst];
        const int y0 = w.dir < 0 ? w.ystart - w.nrows + 1 : w.ystart;
        box[k] = {w.inst, w.x0, std::min(p.nx, w.x0 + L.tx), y0, y0 + w.nrows};
    }
    // [a0, a1) and [b0, b1) meet, with b shifted by -n, 0, +n when periodic
    auto meet = [](int a0, int a1, int b0, int b1, int n, bool periodic) {
        for (int sh = periodic ? -1 : 0; sh <= (periodic ? 1 : 0); ++sh)
            if (b0 + sh * n < a1 && a0 < b1 + sh * n) return true;
        return false;
    };
    std::vector<int> nbr((size_t)L.count * lbm::kMaxNbr, -1);
    for (int k = 0; k < L.count; ++k) {
        const lbm_params& p = c->params[box[k].inst];
        const bool per_y = p.bc_y != LBM_BC_BOUNCEBACK;
        int cnt = 0;
        for (int m = 0; m < L.count; ++m) {
            if (m == k || box[m].inst != box[k].inst) continue;
            if (!meet(box[k].x0 - 2, box[k].x1 + 2, box[m].x0, box[m].x1, p.nx, true)) continue;
            if (!meet(box[k].y0 - 3, box[k].y1 + 3, box[m].y0, box[m].y1, p.ny, per_y)) continue;
            if (cnt == lbm::kMaxNbr) return LBM_OK;   // too many: no persistent launch
            nbr[(size_t)k * lbm::kMaxNbr + cnt++] = m;
        }
    }
    cudaFree(c->d_nbr);
    c->d_nbr = nullptr;
    cudaFree(c->d_multi_done);
    c->d_multi_done = nullptr;
    cudaFree(c->d_mon_multi);
    c->d_mon_multi = nullptr;
    cudaFree(c->d_mon_multi_cnt);
    c->d_mon_multi_cnt = nullptr;
    cudaFree(c->d_mon_multi_sub);
    c->d_mon_multi_sub = nullptr;
    LBM_CK(c, cudaMalloc(&c->d_mon_multi, (size_t)kMultiSteps * L.count * lbm::kMonQ * sizeof(double)));
    LBM_CK(c, cudaMalloc(&c->d_mon_multi_cnt, (size_t)kMultiSteps * c->n * (lbm::kMonSub + 1) * sizeof(int)));
    LBM_CK(c, cudaMalloc(&c->d_mon_multi_sub,
                         (size_t)kMultiSteps * c->n * lbm::kMonSub * lbm::kMonQ * sizeof(double)));
    LBM_CK(c, cudaMalloc(&c->d_nbr, nbr.size() * sizeof(int)));
    LBM_CK(c, cudaMemcpy(c->d_nbr, nbr.data(), nbr.size() * sizeof(int), cudaMemcpyHostToDevice));
    LBM_CK(c, cudaMalloc(&c->d_multi_done, ((size_t)L.count + 1) * sizeof(int)));
    c->multi = true;
    return LBM_OK;
}

// Uploads the work list and sets up the monitor's per-instance item lists.
lbm_status finish_plan(lbm_ctx* c) {
    if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
        c->graph_steps = 0;
    }
    // monitor: per-block slots and, per instance, the list of its work items;
    // each item's position within its instance's list (its sub-group in the
    // monitor's reduction tree) goes into WorkItem::pad
    std::vector<int> csr(c->n + 1 + c->work.size(), 0);
    for (const WorkItem& w : c->work) ++csr[w.inst + 1];
    for (int k = 0; k < c->n; ++k) csr[k + 1] += csr[k];
    {
        std::vector<int> fill(csr.begin(), csr.begin() + c->n);
        for (size_t j = 0; j < c->work.size(); ++j) {
            const int k = c->work[j].inst;
            c->work[j].pad = fill[k] - csr[k];
            csr[c->n + 1 + fill[k]++] = (int)j;
        }
    }
    if (c->d_work) cudaFree(c->d_work);
    c->d_work = nullptr;
    LBM_CK(c, cudaMalloc(&c->d_work, c->work.size() * sizeof(WorkItem)));
    LBM_CK(c, cudaMemcpy(c->d_work, c->work.data(), c->work.size() * sizeof(WorkItem),
                         cudaMemcpyHostToDevice));
    cudaFree(c->d_mon_partials);
    cudaFree(c->d_mon_csr);
    cudaFree(c->d_mon_count);
    cudaFree(c->d_mon_sub);
    c->d_mon_partials = nullptr;
    c->d_mon_csr = nullptr;
    c->d_mon_count = nullptr;
    c->d_mon_sub = nullptr;
    const size_t ncnt = (size_t)c->n * (lbm::kMonSub + 1) * lbm::kCounterStride;
    LBM_CK(c, cudaMalloc(&c->d_mon_partials, c->work.size() * lbm::kMonQ * sizeof(double)));
    LBM_CK(c, cudaMalloc(&c->d_mon_sub, (size_t)c->n * lbm::kMonSub * lbm::kMonQ * sizeof(double)));
    LBM_CK(c, cudaMalloc(&c->d_mon_csr, csr.size() * sizeof(int)));
    LBM_CK(c, cudaMemcpy(c->d_mon_csr, csr.data(), csr.size() * sizeof(int), cudaMemcpyHostToDevice));
    LBM_CK(c, cudaMalloc(&c->d_mon_count, ncnt * sizeof(int)));
    LBM_CK(c, cudaMemset(c->d_mon_count, 0, ncnt * sizeof(int)));
    c->plan_dirty = false;
    return LBM_OK;
}

// D3Q15 work list for the fused march: per instance, tiles of TX x TY columns,
// each split into runs of planes in z; one instance fills one wave (runs sized
// so tiles x runs = SMs x resident blocks), several instances about four waves.
// Neighbouring runs march in opposite directions (halo planes read together).
lbm_status plan_d3(lbm_ctx* c) {
    int tx = 32, ty = 8;
    lbm::march3_tile(&tx, &ty);
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    const int occ = std::max(1, lbm::march3_occupancy(c->form));
    long long tile_planes = 0;
    for (const lbm_params& p : c->params)
        tile_planes += (long long)((p.nx + tx - 1) / tx) * ((p.ny + ty - 1) / ty) * p.nz;
    const int batch_rows =
        (int)std::max<long long>(2, std::min<long long>(64, tile_planes / (4LL * sms * occ)));
    c->work.clear();
    for (int k = 0; k < c->n; ++k) {
        const lbm_params& p = c->params[k];
        const int tiles_x = (p.nx + tx - 1) / tx, tiles_y = (p.ny + ty - 1) / ty;
        int rows = c->rows_req;
        if (rows <= 0) {
            if (c->n == 1) {
                // runs per tile column: least (waves) x (planes a run + 2 for the
                // prologue's four phi and two mu planes), waves counted whole
                const long long target = (long long)sms * occ, tiles = (long long)tiles_x * tiles_y;
                long long best = -1, best_cost = 0;
                for (long long r = 1; r <= p.nz; ++r) {
                    const long long waves = (tiles * r + target - 1) / target;
                    const long long cost = waves * ((p.nz + r - 1) / r + 2);
                    if (best < 0 || cost < best_cost) { best = r; best_cost = cost; }
                }
                rows = (int)((p.nz + best - 1) / best);
            } else {
                rows = batch_rows;
            }
        }
        rows = std::min(rows, p.nz);
        const int nruns = (p.nz + rows - 1) / rows;
        for (int by = 0; by < tiles_y; ++by)
            for (int bx = 0; bx < tiles_x; ++bx)
                for (int r = 0; r < nruns; ++r) {
                    const int z0 = r * rows, z1 = std::min(p.nz, z0 + rows);
                    WorkItem w;
                    w.inst = k;
                    w.x0 = bx * tx;
                    w.pad = by * ty;
                    w.nrows = z1 - z0;
                    w.dir = (r % 2 == 0) ? -1 : 1;
                    w.ystart = w.dir < 0 ? z1 - 1 : z0;
                    c->work.push_back(w);
                }
    }
    c->launches.clear();
    c->launches.push_back({tx, 0, (int)c->work.size(), -1});
    if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
        c->graph_steps = 0;
    }
    if (c->d_work) cudaFree(c->d_work);
    c->d_work = nullptr;
    LBM_CK(c, cudaMalloc(&c->d_work, c->work.size() * sizeof(WorkItem)));
    LBM_CK(c, cudaMemcpy(c->d_work, c->work.data(), c->work.size() * sizeof(WorkItem),
                         cudaMemcpyHostToDevice));
    c->plan_dirty = false;
    return LBM_OK;
}

lbm_status check_instance(lbm_ctx* c, int instance) {
    if (!c) return LBM_EINVAL;
    if (instance < 0 || instance >= c->n) return fail(c, LBM_EINVAL, "instance out of range");
    return LBM_OK;
}

lbm_status sticky(lbm_ctx* c) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "earlier asynchronous work");
    return LBM_OK;
}

// Reads the device status word (synchronises the stream). A bounded device wait
// that ran out leaves LBM_ETIMEOUT there; it stays set (the state is suspect).
lbm_status device_status(lbm_ctx* c) {
    int st = 0;
    cudaError_t e = cudaMemcpyAsync(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "status read-back");
    if (st == lbm::kStatusTimeout) return fail(c, LBM_ETIMEOUT, "a bounded device wait ran out in the step kernel");
    if (st != 0) return fail(c, LBM_ECUDA, "device status word " + std::to_string(st) +
                                                 " (100: a bulk copy was not 16-byte aligned and was skipped)");
    return LBM_OK;
}

lbm_status ensure_out(lbm_ctx* c, size_t cells) {
    if (c->d_out_cells >= cells) return LBM_OK;
    if (c->d_out) cudaFree(c->d_out);
    c->d_out = nullptr;
    c->d_out_cells = 0;
    LBM_CK(c, cudaMalloc(&c->d_out, cells * sizeof(double)));
    c->d_out_cells = cells;
    return LBM_OK;
}

void release(lbm_ctx* c) {
    cudaFree(c->state);
    cudaFree(c->phiu);
    cudaFree(c->sc.phi);
    cudaFree(c->sc.mu);
    cudaFree(c->sc.philo);
    cudaFree(c->d_inst);
    cudaFree(c->d_work);
    cudaFree(c->d_desc);
    cudaFree(c->d_queue);
    cudaFree(c->d_done);
    cudaFree(c->d_nbr);
    cudaFree(c->d_multi_done);
    cudaFree(c->d_mon_multi);
    cudaFree(c->d_mon_multi_cnt);
    cudaFree(c->d_mon_multi_sub);
    cudaFree(c->d_tmp);
    cudaFree(c->d_out);
    cudaFree(c->d_partials);
    cudaFree(c->d_result);
    cudaFree(c->d_status);
    cudaFree(c->d_mon_partials);
    cudaFree(c->d_mon_csr);
    cudaFree(c->d_mon_count);
    cudaFree(c->d_mon_sub);
    cudaFree(c->d_mon);
    cudaFree(c->d_time_base);
    if (c->graph) cudaGraphExecDestroy(c->graph);
    for (cudaStream_t x : c->side) cudaStreamDestroy(x);
    for (cudaEvent_t x : c->join) cudaEventDestroy(x);
    if (c->fork) cudaEventDestroy(c->fork);
    if (c->h_result) cudaFreeHost(c->h_result);
    if (c->h_mon) cudaFreeHost(c->h_mon);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
}

int popcount8(unsigned m) {
    int k = 0;
    for (int b = 0; b < 8; ++b) k += (m >> b) & 1u;
    return k;
}

// valid field masks: the seven D2Q9 fields, plus uz on D3Q15 lattices
bool mask_ok(const lbm_ctx* c, unsigned mask) { return mask != 0 && mask < (c->d3 ? 256u : 128u); }

}  // namespace

extern "C" {

lbm_status lbm_validate_params(const lbm_params* params) {
    if (!params) return LBM_EINVAL;
    return check_params(*params) ? LBM_EINVAL : LBM_OK;
}

lbm_status lbm_create(const lbm_params* params, int n_instances, int precision, void* cuda_stream,
                      lbm_ctx** out) {
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    if (!params || n_instances <= 0) return LBM_EINVAL;
    if (precision < 0 || precision >= kForms) return LBM_EINVAL;
    for (int k = 0; k < n_instances; ++k)
        if (check_params(params[k])) return LBM_EINVAL;
    const bool d3 = is_d3(params[0]);
    for (int k = 0; k < n_instances; ++k)
        if (is_d3(params[k]) != d3) return LBM_EINVAL;   // one lattice a context
    if (d3 && !lbm::d3_form_ok(precision)) return LBM_EINVAL;

    // Instance placement: each instance starts on a 64-cell boundary; the kernels
    // index cells with 32-bit integers, so the padded total must stay below 2^31.
    long long total = 0;
    for (int k = 0; k < n_instances; ++k)
        total += (cells_of(params[k]) + 63) / 64 * 64;
    if (total >= (1LL << 31)) return LBM_EINVAL;

    lbm_ctx* c = new lbm_ctx();
    c->n = n_instances;
    c->form = precision;
    c->d3 = d3;
    c->q = d3 ? 15 : 9;
    c->params.assign(params, params + n_instances);
    c->time.assign(n_instances, 0);
    c->mon_time.assign(n_instances, -1);
    c->ready.assign(n_instances, 0);
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) {
        lbm_status st = cuda_fail(c, e, "cudaGetDevice");
        delete c;
        return st;
    }
    long long base = 0;
    for (int k = 0; k < n_instances; ++k) {
        c->inst.push_back(derive(params[k], base, precision));
        const long long cells = cells_of(params[k]);
        c->max_cells = std::max(c->max_cells, cells);
        base += (cells + 63) / 64 * 64;
    }
    c->S = base;
    auto cleanup = [&](lbm_status st) {
        release(c);
        delete c;
        return st;
    };
    auto alloc = [&](void** p, size_t bytes) { return cudaMalloc(p, bytes); };
    const size_t S = (size_t)c->S;
    {
        auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
        const size_t hb = up(h_planes(precision, c->q) * S * h_elem(precision));
        const size_t h0b = conservative(precision) ? up(S * 2 * sizeof(float)) : 0;
        const size_t gb = up(c->q * S * g_elem(precision));
        const size_t pb = up(S * a_elem(precision));
        c->set_bytes = (long long)(hb + h0b + gb + pb);
        if ((e = alloc(&c->state, 2 * (size_t)c->set_bytes)) != cudaSuccess)
            return cleanup(e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA);
        for (int b = 0; b < 2; ++b) {
            char* set = static_cast<char*>(c->state) + b * c->set_bytes;
            c->h[b] = set;
            c->h0[b] = h0b ? set + hb : nullptr;
            c->g[b] = set + hb + h0b;
            c->p[b] = set + hb + h0b + gb;
        }
    }
    if (d3 && ((e = alloc(&c->sc.phi, S * a_elem(precision))) != cudaSuccess ||
               (e = alloc(&c->sc.mu, S * a_elem(precision))) != cudaSuccess ||
               (conservative(precision) && (e = alloc((void**)&c->sc.philo, S * sizeof(float))) != cudaSuccess)))
        return cleanup(e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA);
    if ((e = alloc(&c->phiu, (d3 ? 3 : 2) * S * a_elem(precision))) != cudaSuccess ||
        (e = alloc((void**)&c->d_inst, n_instances * sizeof(DevInst))) != cudaSuccess ||
        (e = alloc((void**)&c->d_tmp, 2 * (size_t)c->max_cells * sizeof(double))) != cudaSuccess ||
        (e = alloc((void**)&c->d_partials, lbm::kDiagBlocks * lbm::kDiagQuantities * sizeof(double))) !=
            cudaSuccess ||
        (e = alloc((void**)&c->d_result, lbm::kDiagQuantities * sizeof(double))) != cudaSuccess ||
        (e = alloc((void**)&c->d_status, sizeof(int))) != cudaSuccess ||
        (e = alloc((void**)&c->d_time_base, n_instances * sizeof(int64_t))) != cudaSuccess)
        return cleanup(e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA);
    if ((e = cudaMemset(c->d_time_base, 0, n_instances * sizeof(int64_t))) != cudaSuccess)
        return cleanup(LBM_ECUDA);
    if ((e = cudaMemset(c->d_status, 0, sizeof(int))) != cudaSuccess) return cleanup(LBM_ECUDA);
    if ((e = cudaMallocHost((void**)&c->h_result, lbm::kDiagQuantities * sizeof(double))) != cudaSuccess)
        return cleanup(LBM_ENOMEM);
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        if ((e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking)) != cudaSuccess)
            return cleanup(LBM_ECUDA);
        c->own_stream = true;
    }
    if ((e = cudaMemcpy(c->d_inst, c->inst.data(), n_instances * sizeof(DevInst),
                        cudaMemcpyHostToDevice)) != cudaSuccess)
        return cleanup(LBM_ECUDA);
    e = d3 ? lbm::prepare_march3(precision)
           : by_form(precision, [](auto F) { return lbm::prepare_step_t<decltype(F)::value>(); });
    if (e != cudaSuccess) return cleanup(LBM_ECUDA);
    if (plan(c) != LBM_OK) return cleanup(LBM_ECUDA);
    *out = c;
    return LBM_OK;
}

static lbm_status init_common(lbm_ctx* c, int instance, const double* phi0_dev) {
    const lbm_params& p = c->params[instance];
    const int ncells = (int)cells_of(p);
    StepArgs a = step_args(c, 1 - c->cur);   // writes into the current buffers
    cudaError_t e = c->d3 ? lbm::launch_init3(c->form, a, c->sc, instance, ncells, phi0_dev, c->stream)
                          : by_form(c->form, [&](auto F) {
                                return lbm::launch_init_t<decltype(F)::value>(a, phi0_dev, instance, ncells,
                                                                              c->stream);
                            });
    if (e != cudaSuccess) return cuda_fail(c, e, "init kernel");
    c->time[instance] = 0;
    c->mon_time[instance] = -1;
    const int64_t base = -c->steps_total;
    e = cudaMemcpy(c->d_time_base + instance, &base, sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e, "time base upload");
    c->ready[instance] = 1;
    return LBM_OK;
}

lbm_status lbm_init(lbm_ctx* c, int instance, const double* phi0_host) {
    lbm_status st = check_instance(c, instance);
    if (st != LBM_OK) return st;
    if (!phi0_host) return fail(c, LBM_EINVAL, "phi0 is NULL");
    LBM_CK(c, cudaSetDevice(c->device));
    const lbm_params& p = c->params[instance];
    const size_t bytes = (size_t)cells_of(p) * sizeof(double);
    LBM_CK(c, cudaMemcpyAsync(c->d_tmp, phi0_host, bytes, cudaMemcpyHostToDevice, c->stream));
    st = init_common(c, instance, c->d_tmp);
    if (st != LBM_OK) return st;
    // phi0_host is caller-owned: finish reading it before returning
    LBM_CK(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

lbm_status lbm_init_device(lbm_ctx* c, int instance, const double* phi0_device) {
    lbm_status st = check_instance(c, instance);
    if (st != LBM_OK) return st;
    if (!phi0_device) return fail(c, LBM_EINVAL, "phi0 is NULL");
    LBM_CK(c, cudaSetDevice(c->device));
    return init_common(c, instance, phi0_device);
}

namespace {
// lbm_monitor is written on the GPU through its device mirror.
static_assert(sizeof(lbm::MonRecord) == sizeof(lbm_monitor), "monitor record layout");
static_assert(offsetof(lbm::MonRecord, nonfinite) == offsetof(lbm_monitor, nonfinite) &&
                  offsetof(lbm::MonRecord, device_status) == offsetof(lbm_monitor, device_status) &&
                  offsetof(lbm::MonRecord, time) == offsetof(lbm_monitor, time),
              "monitor record layout");

// Queues one launch class of one time step on stream s, reading buffer set `in`.
// With `monitor` its blocks also reduce the per-step monitor; the last block of
// each instance writes that instance's record for time level mon_step.
cudaError_t enqueue_class(lbm_ctx* c, int in, const lbm_ctx::Launch& L, cudaStream_t s, bool monitor,
                          int64_t mon_step = 0) {
    StepArgs a = step_args(c, in);
    a.work = c->d_work + L.offset;
    if (monitor) {
        a.mon = c->d_mon_partials + (long long)L.offset * lbm::kMonQ;
        a.mon_all = c->d_mon_partials;
        a.mon_sub = c->d_mon_sub;
        a.mon_count = c->d_mon_count;
        a.mon_csr = c->d_mon_csr;
        a.mon_n = c->n;
        a.mon_rec = reinterpret_cast<lbm::MonRecord*>(c->d_mon);
        a.time_base = c->d_time_base;
        a.mon_step = mon_step;
        a.mon_host = c->mon_host_dev;
    }
    return by_form(c->form, [&](auto F) {
        return lbm::launch_step_t<decltype(F)::value>(L.tx, a, L.count, s, L.variant, monitor);
    });
}

// D3Q15: the unfused three-kernel step runs under LBM_PIPELINE_PLAIN, and by
// default in FP64, where the fused march is bound by the FP64 pipe and its
// recomputed halo costs more than the scratch planes (647 against 714 MLUPS on
// the 128 x 256 x 128 bubble).
bool d3_unfused(const lbm_ctx* c) {
    return c->pipeline == LBM_PIPELINE_PLAIN || (c->pipeline == LBM_PIPELINE_AUTO && c->form == LBM_F64);
}

// The plan is the one batched launch (step_kernel_x2_batched), which can run
// several steps a launch.
bool batched_plan(const lbm_ctx* c) {
    return !c->d3 && c->launches.size() == 1 && c->launches[0].variant == lbm::kBatched;
}

// Queues `nsteps` steps of a batched plan as one launch, the first reading buffer
// set `in`; wait_extra / wait_limit as in StepArgs (0 / the library's limit).
cudaError_t enqueue_batched(lbm_ctx* c, int in, int nsteps, int wait_extra = 0, int wait_limit = lbm::kWaitLimit) {
    const auto& L = c->launches[0];
    StepArgs a = step_args(c, in);
    a.work = c->d_work + L.offset;
    a.nsteps = nsteps;
    a.wait_extra = wait_extra;
    a.wait_limit = wait_limit;
    return by_form(c->form, [&](auto F) {
        return lbm::launch_step_t<decltype(F)::value>(L.tx, a, L.count, c->stream, L.variant, false);
    });
}

// The plan runs several steps a launch, one block per work item (plan_multi).
bool multi_plan(const lbm_ctx* c) { return c->multi && !c->d3 && c->launches.size() == 1; }

// Queues `nsteps` steps of a persistent plan as one cooperative launch, the
// first reading buffer set `in`, after zeroing the per-item step counters and
// the abort flag; wait_extra / wait_limit as in StepArgs.
// With host_records (device view of pinned host memory; nsteps <= 64) every
// step's monitor record goes there, [step][instance] (the monitor must be on).
cudaError_t enqueue_multi(lbm_ctx* c, int in, int nsteps, int wait_extra = 0, int wait_limit = lbm::kWaitLimit,
                          lbm::MonRecord* host_records = nullptr) {
    const auto& L = c->launches[0];
    cudaError_t e = cudaMemsetAsync(c->d_multi_done, 0, ((size_t)L.count + 1) * sizeof(int), c->stream);
    if (e != cudaSuccess) return e;
    const bool monitor = host_records != nullptr;
    if (monitor) {
        if (nsteps > kMultiSteps || !c->d_mon) return cudaErrorInvalidValue;
        e = cudaMemsetAsync(c->d_mon_multi_cnt, 0, (size_t)nsteps * c->n * (lbm::kMonSub + 1) * sizeof(int),
                            c->stream);
        if (e != cudaSuccess) return e;
    }
    StepArgs a = step_args(c, in);
    a.work = c->d_work + L.offset;
    a.nbr = c->d_nbr;
    a.done = c->d_multi_done;
    a.ndesc = L.count;
    a.nsteps = nsteps;
    a.wait_extra = wait_extra;
    a.wait_limit = wait_limit;
    if (monitor) {
        a.mon = c->d_mon_multi;
        a.mon_sub = c->d_mon_multi_sub;
        a.mon_count = c->d_mon_multi_cnt;
        a.mon_csr = c->d_mon_csr;
        a.mon_n = c->n;
        a.mon_rec = reinterpret_cast<lbm::MonRecord*>(c->d_mon);
        a.time_base = c->d_time_base;
        a.mon_step = c->steps_total;
        a.mon_host = host_records;
    }
    return by_form(c->form, [&](auto F) {
        return lbm::launch_multi_t<decltype(F)::value>(L.tx, a, L.count, c->stream, monitor);
    });
}

// Kernel launches of one directly launched step of the plan.
int step_kernels(const lbm_ctx* c) {
    if (c->d3) return d3_unfused(c) ? 3 * c->n : 1;
    return (int)c->launches.size();
}

// Queues one time step (all launches of the plan) reading buffer set `in`; with
// `monitor` the step kernels also write their monitor slots, reduced per instance.
cudaError_t enqueue_step(lbm_ctx* c, int in, bool monitor = false, int64_t mon_step = 0) {
    if (c->d3) {
        const StepArgs a = step_args(c, in);
        if (d3_unfused(c)) {   // the unfused three-kernel step
            for (int k = 0; k < c->n; ++k) {
                cudaError_t e = lbm::launch_step3(c->form, a, c->sc, k, (int)cells_of(c->params[k]), c->stream);
                if (e != cudaSuccess) return e;
            }
            return cudaSuccess;
        }
        return lbm::launch_march3(c->form, a, c->sc, c->d_work, (int)c->work.size(), c->stream);
    }
    for (const auto& L : c->launches) {
        cudaError_t e = enqueue_class(c, in, L, c->stream, monitor, mon_step);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Captures an even number of steps (starting from parity 0) into a CUDA graph, so
// that long runs of small grids are not bound by launch overhead. With several
// launch classes (strip widths / load paths) each class is its own branch of the
// graph: a class holds whole instances, which depend on nothing else, so its
// steps need not wait for the other classes' -- the classes overlap instead of
// each step ending in the tails of 2-3 short launches. Returns false (and the
// caller launches directly) if the stream cannot be captured: the legacy default
// stream, or a stream the caller is capturing itself.
bool build_graph(lbm_ctx* c) {
    if (c->graph) return true;
    if (!c->use_graphs || c->stream == nullptr || c->stream == cudaStreamLegacy) return false;
    cudaStreamCaptureStatus cs;
    if (cudaStreamIsCapturing(c->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
        return false;
    // about 64 launches a graph
    const int nl = (int)c->launches.size();
    const int per_step = std::max(1, nl);
    const int steps = 2 * std::max(1, 32 / per_step);
    if (nl > 1) {
        while ((int)c->side.size() < nl) {
            cudaStream_t x = nullptr;
            cudaEvent_t ev = nullptr;
            if (cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking) != cudaSuccess) return false;
            c->side.push_back(x);
            if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return false;
            c->join.push_back(ev);
        }
        if (!c->fork && cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming) != cudaSuccess) return false;
    }
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaError_t e = cudaSuccess;
    if (nl > 1) {
        e = cudaEventRecord(c->fork, c->stream);
        for (int i = 0; i < nl && e == cudaSuccess; ++i) {
            e = cudaStreamWaitEvent(c->side[i], c->fork, 0);
            for (int t = 0; t < steps && e == cudaSuccess; ++t)
                e = enqueue_class(c, t & 1, c->launches[i], c->side[i], false);
            if (e == cudaSuccess) e = cudaEventRecord(c->join[i], c->side[i]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->join[i], 0);
        }
    } else if (batched_plan(c)) {
        e = enqueue_batched(c, 0, steps);   // one launch for all the steps
    } else if (multi_plan(c)) {
        e = enqueue_multi(c, 0, steps);     // one launch (after the counters' reset) for all the steps
    } else {
        for (int t = 0; t < steps && e == cudaSuccess; ++t) e = enqueue_step(c, t & 1);
    }
    cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        c->use_graphs = false;
        return false;
    }
    cudaGraphExec_t x = nullptr;
    e = cudaGraphInstantiate(&x, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->use_graphs = false;
        return false;
    }
    c->graph = x;
    c->graph_steps = steps;
    c->graph_launches = nl > 1 ? steps * nl : ((batched_plan(c) || multi_plan(c)) ? 1 : steps * step_kernels(c));
    return true;
}
}  // namespace

lbm_status lbm_step(lbm_ctx* c, int nsteps) {
    if (!c) return LBM_EINVAL;
    if (nsteps < 0) return fail(c, LBM_EINVAL, "nsteps < 0");
    for (int k = 0; k < c->n; ++k)
        if (!c->ready[k]) return fail(c, LBM_ESTATE, "instance not initialised");
    LBM_CK(c, cudaSetDevice(c->device));
    lbm_status st = sticky(c);
    if (st != LBM_OK) return st;
    if (c->plan_dirty && (st = plan(c)) != LBM_OK) return st;
    // with the monitor on, the last step runs the monitored kernels
    const bool mon_last = c->monitor && nsteps > 0;
    int left = mon_last ? nsteps - 1 : nsteps;
    // graph replays cover whole multiples of the captured steps from parity 0
    if (left >= 2 && c->use_graphs) {
        if (c->cur == 1) {
            cudaError_t e = enqueue_step(c, 1);
            if (e != cudaSuccess) return cuda_fail(c, e, "step kernel launch");
            c->step_launches += step_kernels(c);
            c->cur = 0;
            --left;
        }
        if (left >= 2 && build_graph(c)) {
            while (left >= c->graph_steps) {
                cudaError_t e = cudaGraphLaunch(c->graph, c->stream);
                if (e != cudaSuccess) return cuda_fail(c, e, "graph launch");
                c->step_launches += c->graph_launches;
                left -= c->graph_steps;   // even: parity unchanged
            }
        }
    }
    while (left > 0 && (batched_plan(c) || multi_plan(c))) {   // the rest in launches of up to 256 steps
        const int n = std::min(left, 256);
        cudaError_t e = batched_plan(c) ? enqueue_batched(c, c->cur, n) : enqueue_multi(c, c->cur, n);
        if (e != cudaSuccess) return cuda_fail(c, e, "step kernel launch");
        ++c->step_launches;
        c->cur ^= n & 1;
        left -= n;
    }
    for (; left > 0; --left) {
        cudaError_t e = enqueue_step(c, c->cur);
        if (e != cudaSuccess) return cuda_fail(c, e, "step kernel launch");
        c->step_launches += step_kernels(c);
        c->cur ^= 1;
    }
    if (mon_last) {
        // the record's time level is the monitored step's input level
        cudaError_t e = enqueue_step(c, c->cur, true, c->steps_total + nsteps - 1);
        if (e != cudaSuccess) return cuda_fail(c, e, "monitored step launch");
        c->step_launches += step_kernels(c);
        c->cur ^= 1;
    }
    c->steps_total += nsteps;
    for (int k = 0; k < c->n; ++k) {
        c->time[k] += nsteps;
        if (mon_last) c->mon_time[k] = c->time[k] - 1;
    }
    return LBM_OK;
}

lbm_status lbm_step_monitored(lbm_ctx* c, int nsteps, lbm_monitor* host_records) {
    if (!c) return LBM_EINVAL;
    if (nsteps < 1) return fail(c, LBM_EINVAL, "nsteps < 1");
    if (!host_records) return fail(c, LBM_EINVAL, "host_records is NULL");
    if (!c->monitor || !c->d_mon) return fail(c, LBM_ESTATE, "the per-step monitor is off (lbm_set_monitor)");
    LBM_CK(c, cudaSetDevice(c->device));
    void* dptr = nullptr;
    if (cudaHostGetDevicePointer(&dptr, host_records, 0) != cudaSuccess || !dptr) {
        cudaGetLastError();
        return fail(c, LBM_EINVAL, "host_records must be pinned host memory the device can write "
                                   "(cudaMallocHost / cudaHostAlloc)");
    }
    c->mon_host_dev = static_cast<lbm::MonRecord*>(dptr);
    const lbm_status st = lbm_step(c, nsteps);
    c->mon_host_dev = nullptr;
    return st;
}

lbm_status lbm_step_monitored_all(lbm_ctx* c, int nsteps, lbm_monitor* host_records) {
    if (!c) return LBM_EINVAL;
    if (nsteps < 1) return fail(c, LBM_EINVAL, "nsteps < 1");
    if (!host_records) return fail(c, LBM_EINVAL, "host_records is NULL");
    if (!c->monitor || !c->d_mon) return fail(c, LBM_ESTATE, "the per-step monitor is off (lbm_set_monitor)");
    for (int k = 0; k < c->n; ++k)
        if (!c->ready[k]) return fail(c, LBM_ESTATE, "instance not initialised");
    LBM_CK(c, cudaSetDevice(c->device));
    void* dptr = nullptr;
    if (cudaHostGetDevicePointer(&dptr, host_records, 0) != cudaSuccess || !dptr) {
        cudaGetLastError();
        return fail(c, LBM_EINVAL, "host_records must be pinned host memory the device can write "
                                   "(cudaMallocHost / cudaHostAlloc)");
    }
    lbm_status st = sticky(c);
    if (st != LBM_OK) return st;
    if (c->plan_dirty && (st = plan(c)) != LBM_OK) return st;
    lbm::MonRecord* hd = static_cast<lbm::MonRecord*>(dptr);
    for (int done = 0; done < nsteps;) {
        if (multi_plan(c)) {   // up to 64 steps a launch, every step's record from it
            const int k = std::min(nsteps - done, kMultiSteps);
            cudaError_t e = enqueue_multi(c, c->cur, k, 0, lbm::kWaitLimit, hd + (long long)done * c->n);
            if (e != cudaSuccess) return cuda_fail(c, e, "monitored step launch");
            ++c->step_launches;
            c->cur ^= k & 1;
            c->steps_total += k;
            done += k;
        } else {   // one monitored step a launch
            c->mon_host_dev = hd + (long long)done * c->n;
            cudaError_t e = enqueue_step(c, c->cur, true, c->steps_total);
            c->mon_host_dev = nullptr;
            if (e != cudaSuccess) return cuda_fail(c, e, "monitored step launch");
            c->step_launches += step_kernels(c);
            c->cur ^= 1;
            ++c->steps_total;
            ++done;
        }
    }
    for (int k = 0; k < c->n; ++k) {
        c->time[k] += nsteps;
        c->mon_time[k] = c->time[k] - 1;
    }
    return LBM_OK;
}

lbm_status lbm_set_monitor(lbm_ctx* c, int enable) {
    if (!c) return LBM_EINVAL;
    if (c->d3 && enable) return fail(c, LBM_EINVAL, "the per-step monitor serves D2Q9 contexts");
    LBM_CK(c, cudaSetDevice(c->device));
    if (enable && !c->d_mon) {
        LBM_CK(c, cudaMalloc(&c->d_mon, (size_t)c->n * sizeof(lbm_monitor)));
        LBM_CK(c, cudaMallocHost(&c->h_mon, sizeof(lbm_monitor)));
    }
    c->monitor = enable != 0;
    return LBM_OK;
}

lbm_status lbm_read_monitor_async(lbm_ctx* c, int instance, lbm_monitor* host_out) {
    lbm_status st = check_instance(c, instance);
    if (st != LBM_OK) return st;
    if (!host_out) return fail(c, LBM_EINVAL, "out is NULL");
    if (!c->d_mon || c->mon_time[instance] < 0)
        return fail(c, LBM_ESTATE, "no monitored step yet (lbm_set_monitor, then lbm_step)");
    LBM_CK(c, cudaSetDevice(c->device));
    if ((st = sticky(c)) != LBM_OK) return st;
    LBM_CK(c, cudaMemcpyAsync(host_out, c->d_mon + instance, sizeof(lbm_monitor), cudaMemcpyDeviceToHost,
                              c->stream));
    return LBM_OK;
}

lbm_status lbm_read_monitor(lbm_ctx* c, int instance, lbm_monitor* out) {
    lbm_status st = check_instance(c, instance);
    if (st != LBM_OK) return st;
    if (!out) return fail(c, LBM_EINVAL, "out is NULL");
    if (!c->d_mon || c->mon_time[instance] < 0)
        return fail(c, LBM_ESTATE, "no monitored step yet (lbm_set_monitor, then lbm_step)");
    st = lbm_read_monitor_async(c, instance, c->h_mon);
    if (st != LBM_OK) return st;
    LBM_CK(c, cudaStreamSynchronize(c->stream));
    *out = *c->h_mon;
    if (out->device_status != 0) return device_status(c);
    if (out->nonfinite) return fail(c, LBM_ENONFINITE, "non-finite phi or velocity in the monitored step");
    return LBM_OK;
}

lbm_status lbm_set_graphs(lbm_ctx* c, int enable) {
    if (!c) return LBM_EINVAL;
    c->use_graphs = enable != 0;
    if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
        c->graph_steps = 0;
    }
    return LBM_OK;
}

static lbm_status fields_to_device(lbm_ctx* c, int instance, unsigned mask, double* dev_out) {
    const lbm_params& p = c->params[instance];
    if (c->d3) {
        cudaError_t e = lbm::launch_fields3(c->form, step_args(c, c->cur), c->sc, instance, (int)cells_of(p),
                                            mask, dev_out, nullptr, nullptr, c->stream);
        return e == cudaSuccess ? LBM_OK : cuda_fail(c, e, "fields kernels");
    }
    AuxArgs a = aux_args(c, instance);
    a.out = dev_out;
    a.mask = mask;
    cudaError_t e = by_form(c->form, [&](auto F) {
        return lbm::launch_fields_t<decltype(F)::value>(a, p.nx * p.ny, c->stream);
    });
    if (e != cudaSuccess) return cuda_fail(c, e, "fields kernels");
    return LBM_OK;
}

lbm_status lbm_get_fields(lbm_ctx* c, int instance, unsigned mask, double* host_out) {
    lbm_status st = check_instance(c, instance);
    if (st != LBM_OK) return st;
    if (!host_out || !mask_ok(c, mask)) return fail(c, LBM_EINVAL, "bad mask or output");
    if (!c->ready[instance]) return fail(c, LBM_ESTATE, "instance not initialised");
    LBM_CK(c, cudaSetDevice(c->device));
    if ((st = sticky(c)) != LBM_OK) return st;
    const lbm_params& p = c->params[instance];
    const size_t cells = (size_t)cells_of(p) * popcount8(mask);
    if ((st = ensure_out(c, cells)) != LBM_OK) return st;
    if ((st = fields_to_device(c, instance, mask, c->d_out)) != LBM_OK) return st;
    LBM_CK(c, cudaMemcpyAsync(host_out, c->d_out, cells * sizeof(double), cudaMemcpyDeviceToHost,
                              c->stream));
    LBM_CK(c, cudaStreamSynchronize(c->stream));
    return device_status(c);
}

lbm_status lbm_get_fields_device(lbm_ctx* c, int instance, unsigned mask, double* dev_out) {
    lbm_status st = check_instance(c, instance);
    if (st != LBM_OK) return st;
    if (!dev_out || !mask_ok(c, mask)) return fail(c, LBM_EINVAL, "bad mask or output");
    if (!c->ready[instance]) return fail(c, LBM_ESTATE, "instance not initialised");
    LBM_CK(c, cudaSetDevice(c->device));
    if ((st = sticky(c)) != LBM_OK) return st;
    return fields_to_device(c, instance, mask, dev_out);
}

lbm_status lbm_diagnostics(lbm_ctx* c, int instance, lbm_diag* out) {
    lbm_status st = check_instance(c, instance);
    if (st != LBM_OK) return st;
    if (!out) return fail(c, LBM_EINVAL, "out is NULL");
    if (!c->ready[instance]) return fail(c, LBM_ESTATE, "instance not initialised");
    LBM_CK(c, cudaSetDevice(c->device));
    if ((st = sticky(c)) != LBM_OK) return st;
    const lbm_params& p = c->params[instance];
    AuxArgs a = aux_args(c, instance);
    cudaError_t e = c->d3 ? lbm::launch_fields3(c->form, step_args(c, c->cur), c->sc, instance,
                                                (int)cells_of(p), 0u, nullptr, c->d_partials, c->d_result,
                                                c->stream)
                          : by_form(c->form, [&](auto F) {
                                return lbm::launch_diag_t<decltype(F)::value>(a, p.nx * p.ny, c->stream);
                            });
    if (e != cudaSuccess) return cuda_fail(c, e, "diagnostics kernels");
    LBM_CK(c, cudaMemcpyAsync(c->h_result, c->d_result, lbm::kDiagQuantities * sizeof(double),
                              cudaMemcpyDeviceToHost, c->stream));
    LBM_CK(c, cudaStreamSynchronize(c->stream));
    if ((st = device_status(c)) != LBM_OK) return st;
    const double* r = c->h_result;
    std::memset(out, 0, sizeof(*out));
    out->sum_phi = r[0];
    out->sum_rho = r[1];
    out->kinetic_energy = r[2];
    out->max_u = r[3];
    out->mass_A = r[0];
    out->mass_B = r[13];
    out->centroid_A_x = r[4] / r[0];
    out->centroid_A_y = r[5] / r[0];
    out->centroid_B_x = r[6] / r[13];
    out->centroid_B_y = r[7] / r[13];
    out->P_bulk_A = r[9] > 0 ? r[8] / r[9] : 0.0;
    out->n_bulk_A = r[9];
    out->P_bulk_B = r[11] > 0 ? r[10] / r[11] : 0.0;
    out->n_bulk_B = r[11];
    out->nonfinite = r[12] > 0 ? 1 : 0;
    out->time = c->time[instance];
    if (out->nonfinite) return fail(c, LBM_ENONFINITE, "non-finite population");
    return LBM_OK;
}

}  // extern "C"

namespace {
// The state of a context as storage segments (current buffers): h planes, the
// two-float h_0 plane of conservative forms, g planes, phi u, p -- the order of
// checkpoints and of the row exchange.
struct Segment { void* dev; size_t elem; int planes; };

std::vector<Segment> segments(lbm_ctx* c) {
    std::vector<Segment> s;
    s.push_back({c->h[c->cur], h_elem(c->form), h_planes(c->form, c->q)});
    if (conservative(c->form)) s.push_back({c->h0[c->cur], 8, 1});
    s.push_back({c->g[c->cur], g_elem(c->form), c->q});
    s.push_back({c->phiu, a_elem(c->form), c->d3 ? 3 : 2});
    s.push_back({c->p[c->cur], a_elem(c->form), 1});
    return s;
}

// Rows [y0, y0 + nrows) of every state plane of an instance to or from a packed
// device buffer: one 2-D copy per storage segment (pitch = the plane stride).
lbm_status copy_rows(lbm_ctx* c, int instance, int y0, int nrows, void* buf, size_t bytes, bool pack) {
    lbm_status st = check_instance(c, instance);
    if (st != LBM_OK) return st;
    if (!buf) return fail(c, LBM_EINVAL, "row buffer is NULL");
    if (c->d3) return fail(c, LBM_EINVAL, "row exchange serves D2Q9 contexts");
    const lbm_params& p = c->params[instance];
    if (nrows < 1 || y0 < 0 || y0 + nrows > p.ny) return fail(c, LBM_EINVAL, "rows outside the instance");
    if (bytes < (size_t)nrows * lbm_row_bytes(c, instance)) return fail(c, LBM_EINVAL, "row buffer too small");
    LBM_CK(c, cudaSetDevice(c->device));
    const size_t cell0 = (size_t)c->inst[instance].base + (size_t)y0 * p.nx;
    const size_t cells = (size_t)nrows * p.nx;
    unsigned char* b = static_cast<unsigned char*>(buf);
    for (const Segment& sg : segments(c)) {
        unsigned char* plane0 = static_cast<unsigned char*>(sg.dev) + cell0 * sg.elem;
        const size_t width = cells * sg.elem, pitch = (size_t)c->S * sg.elem;
        cudaError_t e = pack ? cudaMemcpy2DAsync(b, width, plane0, pitch, width, sg.planes, cudaMemcpyDeviceToDevice,
                                                 c->stream)
                             : cudaMemcpy2DAsync(plane0, pitch, b, width, width, sg.planes, cudaMemcpyDeviceToDevice,
                                                 c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, pack ? "row pack" : "row unpack");
        b += width * sg.planes;
    }
    return LBM_OK;
}
}  // namespace

extern "C" {

size_t lbm_row_bytes(const lbm_ctx* c, int instance) {
    if (!c || instance < 0 || instance >= c->n || c->d3) return 0;
    size_t per_cell = 0;
    for (const Segment& sg : segments(const_cast<lbm_ctx*>(c))) per_cell += sg.elem * sg.planes;
    return per_cell * (size_t)c->params[instance].nx;
}

lbm_status lbm_pack_rows(lbm_ctx* c, int instance, int y0, int nrows, void* dev_buf, size_t bytes) {
    if (!c) return LBM_EINVAL;
    return copy_rows(c, instance, y0, nrows, dev_buf, bytes, true);
}

lbm_status lbm_unpack_rows(lbm_ctx* c, int instance, int y0, int nrows, const void* dev_buf, size_t bytes) {
    if (!c) return LBM_EINVAL;
    return copy_rows(c, instance, y0, nrows, const_cast<void*>(dev_buf), bytes, false);
}

lbm_status lbm_get_populations(lbm_ctx* c, int instance, double* host_h, double* host_g) {
    lbm_status st = check_instance(c, instance);
    if (st != LBM_OK) return st;
    if (!c->ready[instance]) return fail(c, LBM_ESTATE, "instance not initialised");
    LBM_CK(c, cudaSetDevice(c->device));
    if ((st = sticky(c)) != LBM_OK) return st;
    const lbm_params& p = c->params[instance];
    const size_t n = (size_t)cells_of(p);
    const size_t q = (size_t)c->q;
    if ((st = ensure_out(c, 2 * q * n)) != LBM_OK) return st;
    AuxArgs a = aux_args(c, instance);
    cudaError_t e = c->d3 ? lbm::launch_populations3(c->form, step_args(c, c->cur), c->sc, instance, (int)n,
                                                     c->d_out, c->d_out + q * n, c->stream)
                          : by_form(c->form, [&](auto F) {
                                return lbm::launch_populations_t<decltype(F)::value>(
                                    a, (int)n, c->d_out, c->d_out + 9 * n, c->stream);
                            });
    if (e != cudaSuccess) return cuda_fail(c, e, "populations kernel");
    if (host_h)
        LBM_CK(c, cudaMemcpyAsync(host_h, c->d_out, q * n * sizeof(double), cudaMemcpyDeviceToHost,
                                  c->stream));
    if (host_g)
        LBM_CK(c, cudaMemcpyAsync(host_g, c->d_out + q * n, q * n * sizeof(double),
                                  cudaMemcpyDeviceToHost, c->stream));
    LBM_CK(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

// ---- checkpoints --------------------------------------------------------
namespace {
const char kMagic[8] = {'L', 'B', 'M', 'C', 'K', 'P', 'T', '1'};

bool little_endian() {
    const uint32_t one = 1;
    unsigned char b;
    std::memcpy(&b, &one, 1);
    return b == 1;
}
}  // namespace

lbm_status lbm_save(lbm_ctx* c, const char* path) {
    if (!c || !path) return LBM_EINVAL;
    if (!little_endian()) return fail(c, LBM_EIO, "checkpoints need a little-endian host");
    LBM_CK(c, cudaSetDevice(c->device));
    LBM_CK(c, cudaStreamSynchronize(c->stream));
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(c, LBM_EIO, std::string("cannot open ") + path);
    bool ok = std::fwrite(kMagic, 1, 8, f) == 8;
    const int32_t hdr[4] = {1, c->form, c->n, 0};
    ok = ok && std::fwrite(hdr, sizeof(hdr), 1, f) == 1;
    ok = ok && std::fwrite(c->params.data(), sizeof(lbm_params), c->n, f) == (size_t)c->n;
    ok = ok && std::fwrite(c->time.data(), sizeof(int64_t), c->n, f) == (size_t)c->n;
    std::vector<unsigned char> buf;
    for (const Segment& s : segments(c)) {
        const size_t bytes = (size_t)s.planes * c->S * s.elem;
        buf.resize(bytes);
        cudaError_t e = cudaMemcpy(buf.data(), s.dev, bytes, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            std::fclose(f);
            return cuda_fail(c, e, "checkpoint read-back");
        }
        ok = ok && std::fwrite(buf.data(), 1, bytes, f) == bytes;
    }
    ok = (std::fclose(f) == 0) && ok;
    return ok ? LBM_OK : fail(c, LBM_EIO, std::string("write failed: ") + path);
}

lbm_status lbm_load(lbm_ctx* c, const char* path) {
    if (!c || !path) return LBM_EINVAL;
    if (!little_endian()) return fail(c, LBM_EIO, "checkpoints need a little-endian host");
    LBM_CK(c, cudaSetDevice(c->device));
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(c, LBM_EIO, std::string("cannot open ") + path);
    char magic[8];
    int32_t hdr[4];
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kMagic, 8) == 0;
    ok = ok && std::fread(hdr, sizeof(hdr), 1, f) == 1 && hdr[0] == 1;
    if (!ok) {
        std::fclose(f);
        return fail(c, LBM_EIO, "not a checkpoint file");
    }
    if (hdr[1] != c->form || hdr[2] != c->n) {
        std::fclose(f);
        return fail(c, LBM_EINVAL, "checkpoint precision or instance count differs");
    }
    std::vector<lbm_params> ps(c->n);
    std::vector<int64_t> ts(c->n);
    ok = std::fread(ps.data(), sizeof(lbm_params), c->n, f) == (size_t)c->n &&
         std::fread(ts.data(), sizeof(int64_t), c->n, f) == (size_t)c->n;
    if (!ok || std::memcmp(ps.data(), c->params.data(), sizeof(lbm_params) * c->n) != 0) {
        std::fclose(f);
        return fail(c, ok ? LBM_EINVAL : LBM_EIO, "checkpoint parameters differ");
    }
    LBM_CK(c, cudaStreamSynchronize(c->stream));
    std::vector<unsigned char> buf;
    for (const Segment& s : segments(c)) {
        const size_t bytes = (size_t)s.planes * c->S * s.elem;
        buf.resize(bytes);
        if (std::fread(buf.data(), 1, bytes, f) != bytes) {
            std::fclose(f);
            return fail(c, LBM_EIO, "checkpoint truncated");
        }
        cudaError_t e = cudaMemcpy(s.dev, buf.data(), bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            std::fclose(f);
            return cuda_fail(c, e, "checkpoint upload");
        }
    }
    std::fclose(f);
    c->time = ts;
    c->mon_time.assign(c->n, -1);
    {
        std::vector<int64_t> base(c->n);
        for (int k = 0; k < c->n; ++k) base[k] = c->time[k] - c->steps_total;
        LBM_CK(c, cudaMemcpy(c->d_time_base, base.data(), c->n * sizeof(int64_t), cudaMemcpyHostToDevice));
    }
    c->ready.assign(c->n, 1);
    // the whole state was replaced: a timeout recorded before no longer applies
    LBM_CK(c, cudaMemset(c->d_status, 0, sizeof(int)));
    return LBM_OK;
}

lbm_status lbm_set_launch(lbm_ctx* c, int tile_x, int rows) {
    if (!c) return LBM_EINVAL;
    if (!(tile_x == 0 || tile_x == 32 || tile_x == 64 || tile_x == 128 || tile_x == 256))
        return fail(c, LBM_EINVAL, "tile_x must be 0, 32, 64, 128 or 256");
    if (rows < 0) return fail(c, LBM_EINVAL, "rows must be >= 0");
    c->tile_req = tile_x;
    c->rows_req = rows;
    c->plan_dirty = true;
    return LBM_OK;
}

namespace {
// Tuned launch shapes, per device, storage form and instance-size signature
// (the list of nx, ny, nz, walls of the context's instances), for the life of
// the process: a second context of the same shape takes the shape without trials.
std::mutex g_tune_mutex;
std::map<std::string, lbm_launch_shape> g_tune_cache;

std::string tune_key(const lbm_ctx* c) {
    std::string k = std::to_string(c->device) + "/" + std::to_string(c->form) + "/";
    for (const lbm_params& p : c->params)
        k += std::to_string(p.nx) + "x" + std::to_string(p.ny) + "x" + std::to_string(p.nz) +
             (p.bc_y == LBM_BC_BOUNCEBACK ? "w," : "p,");
    return k;
}

// What one configuration launches: the launch classes (strip width, blocks,
// load path) and the work items; two configurations with the same plan need
// only one trial.
std::string plan_signature(const lbm_ctx* c) {
    std::string sig;
    for (const auto& L : c->launches)
        sig += std::to_string(L.tx) + ":" + std::to_string(L.count) + ":" + std::to_string(L.variant) + ";";
    for (const WorkItem& w : c->work) sig += std::to_string(w.nrows) + ",";
    if (c->multi) sig += "multi";
    return sig;
}
}  // namespace

lbm_status lbm_autotune_shape(lbm_ctx* c, int flags, lbm_launch_shape* out) {
    if (!c) return LBM_EINVAL;
    if (c->d3) return fail(c, LBM_EINVAL, "D3Q15 contexts have no launch shape to tune");
    if (flags & ~LBM_TUNE_NO_CACHE) return fail(c, LBM_EINVAL, "unknown autotune flags");
    for (int k = 0; k < c->n; ++k)
        if (!c->ready[k]) return fail(c, LBM_ESTATE, "instance not initialised");
    LBM_CK(c, cudaSetDevice(c->device));
    lbm_status st = sticky(c);
    if (st != LBM_OK) return st;
    const std::string key = tune_key(c);
    if (!(flags & LBM_TUNE_NO_CACHE)) {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            lbm_launch_shape r = it->second;
            r.trials = 0;
            c->pipeline = r.pipeline;
            c->tile_req = r.tile_x;
            c->rows_req = r.rows;
            c->plan_dirty = true;
            if (out) *out = r;
            return LBM_OK;
        }
    }
    LBM_CK(c, cudaStreamSynchronize(c->stream));
    // Save the state (current buffers) so the trial steps leave no trace.
    std::vector<Segment> segs = segments(c);
    std::vector<void*> saved;
    for (const Segment& sg : segs) {
        void* b = nullptr;
        const size_t bytes = (size_t)sg.planes * c->S * sg.elem;
        cudaError_t e = cudaMalloc(&b, bytes);
        if (e != cudaSuccess) {
            for (void* q : saved) cudaFree(q);
            return cuda_fail(c, e, "autotune backup");
        }
        saved.push_back(b);
        e = cudaMemcpyAsync(b, sg.dev, bytes, cudaMemcpyDeviceToDevice, c->stream);
        if (e != cudaSuccess) {
            for (void* q : saved) cudaFree(q);
            return cuda_fail(c, e, "autotune backup");
        }
    }
    const int cur0 = c->cur;
    const std::vector<int64_t> time0 = c->time;
    const std::vector<int64_t> mon_time0 = c->mon_time;
    const int64_t steps0 = c->steps_total;
    const bool monitor0 = c->monitor;
    const int pipe0 = c->pipeline, tile0 = c->tile_req, rows0 = c->rows_req;
    c->monitor = false;
    // Candidates: load path (two cells a thread in packed FP32, the batched
    // launch, one cell a thread with plain, cp.async or TMA loads), strip width,
    // run length; the built-in plan (AUTO, 0, 0) first.
    struct Cand { int pipe, tile, rows; };
    std::vector<Cand> cands{{LBM_PIPELINE_AUTO, 0, 0}};
    const int pipes[] = {LBM_PIPELINE_PAIRS, LBM_PIPELINE_PERSISTENT, LBM_PIPELINE_BATCHED, LBM_PIPELINE_PLAIN,
                         LBM_PIPELINE_ASYNC,
                         LBM_PIPELINE_TMA};
    const int tiles[] = {0, 64, 128, 256};
    const int rows_c[] = {0, 8, 16, 32, 64};
    for (int pp : pipes)
        for (int tx : tiles)
            for (int r : rows_c) cands.push_back({pp, pp == LBM_PIPELINE_BATCHED ? 0 : tx, r});
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    std::vector<std::string> seen;
    float best = 1e30f, deflt = 0.f;
    Cand bc = cands[0];
    int trials = 0;
    for (const Cand& cd : cands) {
        c->pipeline = cd.pipe;
        c->tile_req = cd.tile;
        c->rows_req = cd.rows;
        c->plan_dirty = true;
        if ((st = plan(c)) != LBM_OK) break;
        const std::string sig = plan_signature(c);
        if (std::find(seen.begin(), seen.end(), sig) != seen.end()) continue;
        seen.push_back(sig);
        ++trials;
        // warm-up (captures the graph of this plan), then the best of three timings
        // of whole graph replays from buffer parity 0 -- the way lbm_step runs long
        // step counts: a plan of several launch classes runs them as concurrent
        // graph branches there, one after the other in direct launches
        if (c->cur == 1 && (st = lbm_step(c, 1)) != LBM_OK) break;
        if ((st = lbm_step(c, 2)) != LBM_OK) break;
        const int nt = std::max(8, c->use_graphs && c->graph ? c->graph_steps : 0);
        float ms = 1e30f;
        for (int rep = 0; rep < 3 && st == LBM_OK; ++rep) {
            cudaEventRecord(e0, c->stream);
            st = lbm_step(c, nt);
            cudaEventRecord(e1, c->stream);
            cudaEventSynchronize(e1);
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            ms = std::min(ms, t / (float)nt);
        }
        if (st != LBM_OK) break;
        if (trials == 1) deflt = ms;
        if (ms < best) {
            best = ms;
            bc = cd;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // Restore the state, the clocks and the monitor exactly as they were.
    c->cur = cur0;
    segs = segments(c);
    for (size_t k = 0; k < segs.size(); ++k)
        cudaMemcpyAsync(segs[k].dev, saved[k], (size_t)segs[k].planes * c->S * segs[k].elem,
                        cudaMemcpyDeviceToDevice, c->stream);
    cudaError_t se = cudaStreamSynchronize(c->stream);
    for (void* q : saved) cudaFree(q);
    c->time = time0;
    c->mon_time = mon_time0;
    c->monitor = monitor0;
    if (st == LBM_OK && se != cudaSuccess) st = cuda_fail(c, se, "autotune restore");
    if (c->steps_total != steps0) {   // the device time base counts from steps_total
        std::vector<int64_t> base(c->n);
        for (int k = 0; k < c->n; ++k) base[k] = c->time[k] - steps0;
        c->steps_total = steps0;
        if (cudaMemcpy(c->d_time_base, base.data(), c->n * sizeof(int64_t), cudaMemcpyHostToDevice) != cudaSuccess &&
            st == LBM_OK)
            st = fail(c, LBM_ECUDA, "autotune: time base restore");
    }
    if (st != LBM_OK) {
        c->pipeline = pipe0;
        c->tile_req = tile0;
        c->rows_req = rows0;
        c->plan_dirty = true;
        return st;
    }
    c->pipeline = bc.pipe;
    c->tile_req = bc.tile;
    c->rows_req = bc.rows;
    c->plan_dirty = true;
    lbm_launch_shape r;
    r.pipeline = bc.pipe;
    r.tile_x = bc.tile;
    r.rows = bc.rows;
    r.trials = trials;
    r.ms_per_step = best;
    r.default_ms_per_step = deflt;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tune_cache[key] = r;
    }
    if (out) *out = r;
    return sticky(c);
}

lbm_status lbm_autotune(lbm_ctx* c, int* best_tile_x, int* best_rows) {
    lbm_launch_shape r;
    lbm_status st = lbm_autotune_shape(c, LBM_TUNE_NO_CACHE, &r);
    if (st != LBM_OK) return st;
    if (best_tile_x) *best_tile_x = r.tile_x;
    if (best_rows) *best_rows = r.rows;
    return LBM_OK;
}

long long lbm_step_launch_count(const lbm_ctx* c) { return c ? c->step_launches : 0; }

int lbm_launches_per_step(const lbm_ctx* c) {
    if (!c) return 0;
    if (c->plan_dirty) {
        lbm_ctx* m = const_cast<lbm_ctx*>(c);
        if (cudaSetDevice(m->device) != cudaSuccess || plan(m) != LBM_OK) return 0;
    }
    return (c->d3 && d3_unfused(c)) ? 3 * c->n : (int)c->launches.size();
}

int64_t lbm_time(const lbm_ctx* c, int instance) {
    if (!c || instance < 0 || instance >= c->n) return -1;
    return c->time[instance];
}

namespace {

// One thread arms an mbarrier for 16 bytes that no copy will ever deliver and
// waits on it with the step kernel's bounded wait; when the wait gives up it
// records the timeout in the status word, as the step kernel does.
__global__ void wait_timeout_kernel(int rounds, int* status) {
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x != 0) return;
    const uint32_t b = lbm::smem_u32(&bar);
    lbm::mbar_init(b, 1);
    lbm::fence_mbar_init();
    lbm::mbar_expect_tx(b, 16);
    if (!lbm::mbar_wait(b, 0, rounds)) atomicExch(status, lbm::kStatusTimeout);
}

}  // namespace

lbm_status lbm_inject_batched_wait_timeout(lbm_ctx* c, int rounds) {
    if (!c) return LBM_EINVAL;
    if (rounds < 1 || rounds > lbm::kWaitLimit)
        return fail(c, LBM_EINVAL, "rounds must be in 1 .. 2^21");
    for (int k = 0; k < c->n; ++k)
        if (!c->ready[k]) return fail(c, LBM_ESTATE, "instance not initialised");
    LBM_CK(c, cudaSetDevice(c->device));
    lbm_status st = sticky(c);
    if (st != LBM_OK) return st;
    if (c->plan_dirty && (st = plan(c)) != LBM_OK) return st;
    if (!batched_plan(c) && !multi_plan(c))
        return fail(c, LBM_ESTATE, "the context runs neither the batched nor the persistent launch");
    // two steps; every item of the second waits for one finished item (batched)
    // or step (persistent) more than there are, so each of those waits runs out
    // after `rounds` rounds
    LBM_CK(c, batched_plan(c) ? enqueue_batched(c, c->cur, 2, 1, rounds) : enqueue_multi(c, c->cur, 2, 1, rounds));
    return LBM_OK;
}

lbm_status lbm_inject_wait_timeout(lbm_ctx* c, int rounds) {
    if (!c) return LBM_EINVAL;
    if (rounds < 1 || rounds > lbm::kWaitLimit)
        return fail(c, LBM_EINVAL, "rounds must be in 1 .. 2^21");
    LBM_CK(c, cudaSetDevice(c->device));
    wait_timeout_kernel<<<1, 32, 0, c->stream>>>(rounds, c->d_status);
    LBM_CK(c, cudaGetLastError());
    return LBM_OK;
}

lbm_status lbm_sync(lbm_ctx* c) {
    if (!c) return LBM_EINVAL;
    LBM_CK(c, cudaSetDevice(c->device));
    LBM_CK(c, cudaStreamSynchronize(c->stream));
    lbm_status st = sticky(c);
    return st != LBM_OK ? st : device_status(c);
}

lbm_status lbm_set_pipeline(lbm_ctx* c, int mode) {
    if (!c) return LBM_EINVAL;
    if (mode < LBM_PIPELINE_AUTO || mode > LBM_PIPELINE_PERSISTENT)
        return fail(c, LBM_EINVAL, "pipeline mode must be one of LBM_PIPELINE_*");
    c->pipeline = mode;
    c->plan_dirty = true;
    return LBM_OK;
}

lbm_status lbm_launch_info(lbm_ctx* c, int index, int* tile_x, int* blocks, int* variant) {
    if (!c) return LBM_EINVAL;
    if (c->d3) return fail(c, LBM_EINVAL, "D3Q15 contexts launch three fixed kernels an instance");
    if (c->plan_dirty) {
        LBM_CK(c, cudaSetDevice(c->device));
        lbm_status st = plan(c);
        if (st != LBM_OK) return st;
    }
    if (index < 0 || index >= (int)c->launches.size()) return fail(c, LBM_EINVAL, "launch index out of range");
    const auto& L = c->launches[index];
    if (tile_x) *tile_x = L.tx;
    if (blocks) *blocks = L.count;
    if (variant) *variant = L.variant;
    return LBM_OK;
}

const char* lbm_last_error(const lbm_ctx* c) { return c ? c->err.c_str() : "null context"; }

void lbm_destroy(lbm_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    release(c);
    delete c;
}

}  // extern "C"
