// lbm_internal.h -- types shared by the host API and the kernel translation units.
// Not part of the public ABI (include/lbm.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

// Per-instance constants, derived on the host from lbm_params (Eqs. 6-7, 17,
// gamma of Sec. 3.2.1), read once per thread block.
struct DevInst {
    long long base;          // first cell of the instance inside every SoA plane
    int nx, ny;
    int nz;                  // D3Q15 contexts: planes in z (periodic); 1 for D2Q9
    int walls;               // 1: halfway bounce-back walls in y
    int qim;                 // 1: S1 = -gamma M lap(mu)
    int pscheme;             // LBM_P_*
    int sforce;              // LBM_FS_*
    int visc;                // LBM_VISC_*
    int uniform_nu;          // 1: inverse-linear model with nu_A = nu_B (tau_g constant)
    double rho_A, rho_B, drho;       // drho = (rho_A - rho_B) / (phi_A - phi_B)
    double inv_nu_A, inv_nu_B;       // inverse-linear viscosity
    double mu_A, mu_B;               // dynamic viscosities rho nu (step model)
    double beta, kappa, eta;
    double gammaM;                   // gamma * M_phi
    double inv_tau_h;
    double force_x, force_y, gravity;
    double h_scale, g_scale;         // storage scales of reduced-precision forms (powers of 2)
    double tgm0, inv_tau_g0;         // tau_g - 1/2 and 1/tau_g for uniform_nu
};

// One thread block's work: a strip of columns [x0, x0 + TX) (clipped to nx) of
// one instance, marching over nrows rows from ystart in direction dir (+1/-1).
struct WorkItem {
    int inst, x0, ystart, nrows, dir, pad;   // pad: D2Q9, the item's position within its
                                             // instance's items; D3Q15, the tile's y0
};

// A block's share of the batched step (step_kernel_x2_batched): one work item
// of up to 256 columns that all 128 threads march (item[1] == kDescWide), or two
// of up to 128 columns that two groups of 64 threads march side by side (an
// unused entry is -1).
constexpr int kDescWide = -2;
// the persistent multi-step plan (step_kernel_x2_multi): neighbour items an item
constexpr int kMaxNbr = 8;
struct BlockDesc {
    int item[2];
};

// Device buffers of one step (ping-pong: *_in is time t, *_out time t + 1).
struct StepArgs {
    const void* h_in;  void* h_out;     // 9 planes (h_1..h_8 only for conservative forms)
    const void* h0_in; void* h0_out;    // conservative forms: h_0 as float2 (hi, lo), else null
    const void* g_in;  void* g_out;     // 9 planes
    void* phiu;                         // 2 planes, updated in place
    const void* p_in;  void* p_out;     // 1 plane each
    long long S;                        // plane stride in cells
    const DevInst* inst;
    const WorkItem* work;
    int* status;                        // device status word (0 = ok), see kStatusTimeout
    double* mon;                        // monitor: kMonQ doubles per block of this launch
    // Per-step monitor, final reduction (kernels with the monitor only), a
    // two-level tree: a block stores its slot and counts itself in the counter
    // of its sub-group (its position within the instance's items modulo
    // kMonSub); the last block of a sub-group adds the sub-group's slots into a
    // sub-slot and counts itself at the instance level; the last of those adds
    // the sub-slots and writes the record. Counters go back to zero as used.
    double* mon_all;                    // slots of every work item of the plan
    double* mon_sub;                    // kMonSub sub-slots (kMonQ doubles) per instance
    int* mon_count;                     // per instance: kMonSub + 1 counters, kCounterStride ints apart
    const int* mon_csr;                 // per instance k: items idx[csr[k] .. csr[k+1]) (idx at csr + n + 1)
    int mon_n;                          // instances
    struct MonRecord* mon_rec;          // one record per instance
    struct MonRecord* mon_host;         // optional: caller's pinned host records (device-mapped), or null
    const int64_t* time_base;           // per instance: time level - steps of the context
    long long mon_step;                 // steps of the context before the monitored step
    // batched step only: block descriptors, their number, and the queue
    // counters {next (step, descriptor), blocks finished, abort} (zero between
    // launches). One launch runs nsteps steps: step s reads the buffers above
    // when s is even, the *_out ones when s is odd, and an item of step s > 0
    // first waits (bounded: wait_limit rounds) until done[inst], the items of
    // its instance finished in this launch, reaches s x (items_csr[inst + 1] -
    // items_csr[inst]) + wait_extra (0; a test sets 1 to make the wait run out).
    const BlockDesc* desc;
    int ndesc;
    int* queue;
    int* done;
    const int* items_csr;
    const int* nbr;        // persistent multi-step plan: kMaxNbr neighbour items per item, -1 padded
    long long set_delta;   // bytes from each *_in array to its *_out array (the same for all)
    int ninst;
    int nsteps;
    int wait_limit;
    int wait_extra;
};

// Device layout of lbm_monitor (include/lbm.h; the host checks size and offsets).
struct MonRecord {
    double sum_phi, kinetic_energy, max_u;
    int32_t nonfinite, device_status;
    int64_t time;
};

// Doubles a block of a monitored step writes: sum phi, kinetic energy,
// max |u|^2, non-finite flag.
constexpr int kMonQ = 4;
// Sub-groups of an instance's blocks in the monitor's reduction tree, and the
// spacing of its counters (one 128-byte line each: the atomics of different
// counters do not queue on one address).
constexpr int kMonSub = 8;
constexpr int kCounterStride = 32;

// Value a kernel writes to the status word when a bounded device wait runs out
// (equal to LBM_ETIMEOUT of include/lbm.h).
constexpr int kStatusTimeout = 5;

// Buffers of the macroscopic / diagnostic kernels.
struct AuxArgs {
    const void* h; const void* h0; const void* g; const void* phiu; const void* p_prev;
    long long S;
    const DevInst* inst;
    int instance;
    double* tmp_phi;      // nx*ny scratch
    double* tmp_mu;       // nx*ny scratch
    double* out;          // field outputs (fields kernel)
    unsigned mask;
    double* partials;     // diagnostics: per-block partial sums
    double* result;       // diagnostics: final record
};

constexpr int kDiagQuantities = 14;   // quantities of diag_pass (lbm_device.cuh)
constexpr int kDiagBlocks = 304;      // 2 x 152 SMs

// Launchers, instantiated once per storage form in lbm_form<N>.cu.
// Step kernel variants: synchronous loads; per-thread cp.async prefetch (FP32
// storage of h and p); bulk copies by the TMA (FP32 arithmetic, 16-byte rows);
// two cells per thread in packed FP32 (FP32 arithmetic, nx even, tile >= 64).
// kBatched: the pairs kernel over every instance in one persistent launch
// (block descriptors of two 128-column strips).
enum StepVariant { kPlain = 0, kAsync = 1, kTma = 2, kPairs = 3, kBatched = 4 };
template <int FORM> cudaError_t launch_step_t(int tile_x, const StepArgs& a, int nwork, cudaStream_t s,
                                              int variant, bool monitor);
template <int FORM> cudaError_t prepare_step_t();          // opt-in shared memory sizes
template <int FORM> size_t step_smem_t(int tile_x);
template <int FORM> int batched_occupancy_t();             // resident blocks per SM, batched kernel
// several steps of a paired plan in one cooperative launch, and its residency
template <int FORM> cudaError_t launch_multi_t(int tile_x, const StepArgs& a, int nwork, cudaStream_t s,
                                               bool monitor);
template <int FORM> int multi_occupancy_t(int tile_x);
template <int FORM> int step_occupancy_t(int tile_x, int variant);   // resident blocks per SM
template <int FORM> bool has_tma_t();                      // the form has a TMA-fed kernel
template <int FORM> bool has_async_t();                    // the form has the cp.async kernel
template <int FORM> bool has_pairs_t();                    // the form has the paired kernel
template <int FORM> cudaError_t launch_init_t(const StepArgs& a, const double* phi0, int instance,
                                              int ncells, cudaStream_t s);
template <int FORM> cudaError_t launch_fields_t(const AuxArgs& a, int ncells, cudaStream_t s);
template <int FORM> cudaError_t launch_diag_t(const AuxArgs& a, int ncells, cudaStream_t s);
template <int FORM> cudaError_t launch_populations_t(const AuxArgs& a, int ncells, double* out_h,
                                                     double* out_g, cudaStream_t s);

// ---- D3Q15 (lbm_d3q15.cu): three kernels a step over each instance's cells.
// Scratch planes of a 3-D context: phi and mu in the arithmetic type, the low
// part of phi (conservative form) in FP32.
struct D3Scratch {
    void* phi;
    void* mu;
    float* philo;
};
bool d3_form_ok(int form);   // FP64, FP32, FP32 with the two-float h_0
// unfused step (phi, mu, collide kernels) of one instance
cudaError_t launch_step3(int form, const StepArgs& s, const D3Scratch& x, int instance, int ncells,
                         cudaStream_t st);
// fused step: one launch over a work list of (instance, x0, y0 = pad, z run)
// items, tiles of march3_tile() columns
void march3_tile(int* tx, int* ty);
cudaError_t prepare_march3(int form);
int march3_occupancy(int form);
cudaError_t launch_march3(int form, const StepArgs& s, const D3Scratch& x, const WorkItem* work, int nwork,
                          cudaStream_t st);
cudaError_t launch_init3(int form, const StepArgs& s, const D3Scratch& x, int instance, int ncells,
                         const double* phi0, cudaStream_t st);
// fields (mask bits: phi, ux, uy, p, rho, mu, P, uz) into out (may be null) and,
// with partials, the kDiagQuantities diagnostics into result
cudaError_t launch_fields3(int form, const StepArgs& s, const D3Scratch& x, int instance, int ncells,
                           unsigned mask, double* out, double* partials, double* result, cudaStream_t st);
cudaError_t launch_populations3(int form, const StepArgs& s, const D3Scratch& x, int instance, int ncells,
                                double* out_h, double* out_g, cudaStream_t st);

}  // namespace lbm
