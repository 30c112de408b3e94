// lbm_launch.cuh -- host-side launchers of the kernels of one storage form.
// Included by lbm_form<N>.cu, which instantiates them for its form.
#pragma once

#include "lbm_aux.cuh"
#include "lbm_device.cuh"
#include "lbm_step_tma.cuh"
#include "lbm_step_x2.cuh"

namespace lbm {

template <int FORM>
constexpr bool kHasTma = sizeof(typename Form<FORM>::R) == 4;

template <int FORM>
bool has_tma_t() { return kHasTma<FORM>; }

template <int FORM>
bool has_async_t() { return kAsyncOk<FORM>; }

template <int FORM>
bool has_pairs_t() { return kHasTma<FORM>; }   // the FP32-arithmetic forms

// paired kernel: tile_x columns per block, tile_x / 2 threads
template <int FORM, int TX>
static cudaError_t launch_pairs_tx(const StepArgs& a, int nwork, cudaStream_t s, bool monitor) {
    if (monitor) step_kernel_x2<FORM, TX, true><<<nwork, TX, X2Smem<FORM, TX>::bytes, s>>>(a);
    else step_kernel_x2<FORM, TX><<<nwork, TX, X2Smem<FORM, TX>::bytes, s>>>(a);
    return cudaGetLastError();
}

// variant: kPlain (synchronous loads), kAsync (per-thread cp.async prefetch),
// kTma (bulk copies); the caller only asks for a variant the form has. A
// monitored step always runs the synchronous-load kernel with the monitor.
template <int FORM, int TX>
static cudaError_t launch_step_tx(const StepArgs& a, int nwork, cudaStream_t s, int variant, bool monitor) {
    if (monitor) {
        step_kernel<FORM, TX, false, true><<<nwork, TX, StepSmem<FORM, TX>::bytes, s>>>(a);
        return cudaGetLastError();
    }
    if constexpr (kHasTma<FORM>) {
        if (variant == kTma) {
            step_kernel_tma<FORM, TX><<<nwork, TX, TmaSmem<FORM, TX>::bytes, s>>>(a);
            return cudaGetLastError();
        }
    }
    if constexpr (kAsyncOk<FORM>) {
        if (variant == kAsync) {
            step_kernel<FORM, TX, true><<<nwork, TX, StepSmem<FORM, TX>::bytes, s>>>(a);
            return cudaGetLastError();
        }
    }
    step_kernel<FORM, TX, false><<<nwork, TX, StepSmem<FORM, TX>::bytes, s>>>(a);
    return cudaGetLastError();
}

template <int FORM>
cudaError_t launch_step_t(int tile_x, const StepArgs& a, int nwork, cudaStream_t s, int variant,
                          bool monitor) {
    if (nwork <= 0) return cudaSuccess;
    if (monitor && a.mon == nullptr) return cudaErrorInvalidValue;
    if constexpr (kHasTma<FORM>) {
        if (variant == kBatched) {   // nwork = blocks of the persistent grid (at most those resident)
            if (a.desc == nullptr || a.queue == nullptr || a.done == nullptr) return cudaErrorInvalidValue;
            if (monitor) {
                if (a.nsteps != 1) return cudaErrorInvalidValue;
                step_kernel_x2_batched<FORM, true><<<nwork, 128, X2Batched<FORM>::bytes, s>>>(a);
                return cudaGetLastError();
            }
            // several steps: the blocks wait on one another's items, so the grid
            // is launched cooperatively (all of it resident at once)
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(nwork);
            cfg.blockDim = dim3(128);
            cfg.dynamicSmemBytes = X2Batched<FORM>::bytes;
            cfg.stream = s;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeCooperative;
            attr[0].val.cooperative = a.nsteps > 1 ? 1 : 0;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            return cudaLaunchKernelEx(&cfg, step_kernel_x2_batched<FORM, false>, a);
        }
        if (variant == kPairs) {
            switch (tile_x) {
                case 64: return launch_pairs_tx<FORM, 32>(a, nwork, s, monitor);
                case 128: return launch_pairs_tx<FORM, 64>(a, nwork, s, monitor);
                case 256: return launch_pairs_tx<FORM, 128>(a, nwork, s, monitor);
                default: return cudaErrorInvalidValue;
            }
        }
    }
    switch (tile_x) {
        case 32: return launch_step_tx<FORM, 32>(a, nwork, s, variant, monitor);
        case 64: return launch_step_tx<FORM, 64>(a, nwork, s, variant, monitor);
        case 128: return launch_step_tx<FORM, 128>(a, nwork, s, variant, monitor);
        case 256: return launch_step_tx<FORM, 256>(a, nwork, s, variant, monitor);
        default: return cudaErrorInvalidValue;
    }
}

template <int FORM, int TX>
static cudaError_t prep_tx() {
    cudaError_t e = cudaFuncSetAttribute(step_kernel<FORM, TX, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)StepSmem<FORM, TX>::bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(step_kernel<FORM, TX, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)StepSmem<FORM, TX>::bytes);
    if constexpr (kAsyncOk<FORM>) {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(step_kernel<FORM, TX, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)StepSmem<FORM, TX>::bytes);
    }
    if constexpr (kHasTma<FORM>) {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(step_kernel_tma<FORM, TX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)TmaSmem<FORM, TX>::bytes);
        if constexpr (TX >= 32 && TX <= 128) {   // paired kernel: 64..256 columns
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(step_kernel_x2<FORM, TX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)X2Smem<FORM, TX>::bytes);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(step_kernel_x2<FORM, TX, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)X2Smem<FORM, TX>::bytes);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(step_kernel_x2_multi<FORM, TX>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)X2Smem<FORM, TX>::bytes);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(step_kernel_x2_multi<FORM, TX, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)X2Smem<FORM, TX>::bytes);
        }
    }
    return e;
}

template <int FORM>
cudaError_t prepare_step_t() {
    cudaError_t e;
    if ((e = prep_tx<FORM, 32>()) != cudaSuccess) return e;
    if ((e = prep_tx<FORM, 64>()) != cudaSuccess) return e;
    if ((e = prep_tx<FORM, 128>()) != cudaSuccess) return e;
    if ((e = prep_tx<FORM, 256>()) != cudaSuccess) return e;
    if constexpr (kHasTma<FORM>) {
        e = cudaFuncSetAttribute(step_kernel_x2_batched<FORM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)X2Batched<FORM>::bytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(step_kernel_x2_batched<FORM, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)X2Batched<FORM>::bytes);
    }
    return e;
}

template <int FORM>
int batched_occupancy_t() {
    if constexpr (kHasTma<FORM>) {
        int n = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel_x2_batched<FORM>, 128,
                                                                      X2Batched<FORM>::bytes);
        return e == cudaSuccess ? n : 0;
    }
    return 0;
}

// Several steps of a paired plan in one cooperative launch (step_kernel_x2_multi):
// nwork items = blocks, all resident (the caller checks multi_occupancy_t).
template <int FORM, int TX>
static cudaError_t launch_multi_tx(const StepArgs& a, int nwork, cudaStream_t s, bool monitor) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nwork);
    cfg.blockDim = dim3(TX);
    cfg.dynamicSmemBytes = X2Smem<FORM, TX>::bytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (monitor) return cudaLaunchKernelEx(&cfg, step_kernel_x2_multi<FORM, TX, true>, a);
    return cudaLaunchKernelEx(&cfg, step_kernel_x2_multi<FORM, TX>, a);
}

template <int FORM>
cudaError_t launch_multi_t(int tile_x, const StepArgs& a, int nwork, cudaStream_t s, bool monitor) {
    if constexpr (kHasTma<FORM>) {
        if (nwork <= 0) return cudaSuccess;
        if (a.nbr == nullptr || a.done == nullptr) return cudaErrorInvalidValue;
        if (monitor && (a.mon == nullptr || a.mon_count == nullptr || a.mon_csr == nullptr)) return cudaErrorInvalidValue;
        switch (tile_x) {
            case 64: return launch_multi_tx<FORM, 32>(a, nwork, s, monitor);
            case 128: return launch_multi_tx<FORM, 64>(a, nwork, s, monitor);
            case 256: return launch_multi_tx<FORM, 128>(a, nwork, s, monitor);
            default: return cudaErrorInvalidValue;
        }
    }
    return cudaErrorInvalidValue;
}

// resident blocks per SM of the multi-step paired kernel for a strip width
template <int FORM>
int multi_occupancy_t(int tile_x) {
    int n = 0;
    if constexpr (kHasTma<FORM>) {
        cudaError_t e = cudaErrorInvalidValue;
        switch (tile_x) {
            case 64:
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel_x2_multi<FORM, 32>, 32,
                                                                  X2Smem<FORM, 32>::bytes);
                break;
            case 128:
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel_x2_multi<FORM, 64>, 64,
                                                                  X2Smem<FORM, 64>::bytes);
                break;
            case 256:
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel_x2_multi<FORM, 128>, 128,
                                                                  X2Smem<FORM, 128>::bytes);
                break;
            default: break;
        }
        if (e != cudaSuccess) n = 0;
    }
    return n;
}

template <int FORM>
size_t step_smem_t(int tile_x) {
    switch (tile_x) {
        case 32: return StepSmem<FORM, 32>::bytes;
        case 64: return StepSmem<FORM, 64>::bytes;
        case 128: return StepSmem<FORM, 128>::bytes;
        case 256: return StepSmem<FORM, 256>::bytes;
        default: return 0;
    }
}

template <int FORM, int TX>
static int occ_tx(int variant) {
    int n = 0;
    cudaError_t e;
    if constexpr (kHasTma<FORM>) {
        if (variant == kPairs) {
            if constexpr (TX >= 64) {
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel_x2<FORM, TX / 2>, TX / 2,
                                                                  X2Smem<FORM, TX / 2>::bytes);
                return e == cudaSuccess ? n : 0;
            }
            return 0;
        }
    }
    if constexpr (kHasTma<FORM>) {
        if (variant == kTma) {
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel_tma<FORM, TX>, TX,
                                                              TmaSmem<FORM, TX>::bytes);
            return e == cudaSuccess ? n : 0;
        }
    }
    if constexpr (kAsyncOk<FORM>) {
        if (variant == kAsync) {
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel<FORM, TX, true>, TX,
                                                              StepSmem<FORM, TX>::bytes);
            return e == cudaSuccess ? n : 0;
        }
    }
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel<FORM, TX, false>, TX,
                                                      StepSmem<FORM, TX>::bytes);
    return e == cudaSuccess ? n : 0;
}

template <int FORM>
int step_occupancy_t(int tile_x, int variant) {
    switch (tile_x) {
        case 32: return occ_tx<FORM, 32>(variant);
        case 64: return occ_tx<FORM, 64>(variant);
        case 128: return occ_tx<FORM, 128>(variant);
        case 256: return occ_tx<FORM, 256>(variant);
        default: return 0;
    }
}

static inline int grid_for(int ncells, int block) {
    int g = (ncells + block - 1) / block;
    return g < 1 ? 1 : (g > 8 * 152 ? 8 * 152 : g);
}

template <int FORM>
cudaError_t launch_init_t(const StepArgs& a, const double* phi0, int instance, int ncells,
                          cudaStream_t s) {
    init_kernel<FORM><<<grid_for(ncells, 256), 256, 0, s>>>(a, phi0, instance);
    return cudaGetLastError();
}

template <int FORM>
cudaError_t launch_fields_t(const AuxArgs& a, int ncells, cudaStream_t s) {
    const int g = grid_for(ncells, 256);
    phi_pass<FORM><<<g, 256, 0, s>>>(a);
    mu_pass<FORM><<<g, 256, 0, s>>>(a);
    fields_pass<FORM><<<g, 256, 0, s>>>(a);
    return cudaGetLastError();
}

template <int FORM>
cudaError_t launch_diag_t(const AuxArgs& a, int ncells, cudaStream_t s) {
    const int g = grid_for(ncells, 256);
    phi_pass<FORM><<<g, 256, 0, s>>>(a);
    mu_pass<FORM><<<g, 256, 0, s>>>(a);
    diag_pass<FORM><<<kDiagBlocks, 256, 0, s>>>(a);
    diag_final<<<1, kDiagFinalThreads, 0, s>>>(a.partials, kDiagBlocks, a.result);
    return cudaGetLastError();
}

template <int FORM>
cudaError_t launch_populations_t(const AuxArgs& a, int ncells, double* out_h, double* out_g,
                                 cudaStream_t s) {
    populations_pass<FORM><<<grid_for(ncells, 256), 256, 0, s>>>(a, out_h, out_g);
    return cudaGetLastError();
}

#define LBM_INSTANTIATE_FORM(F)                                                               \
    template cudaError_t launch_step_t<F>(int, const StepArgs&, int, cudaStream_t, int, bool); \
    template cudaError_t prepare_step_t<F>();                                                 \
    template size_t step_smem_t<F>(int);                                                      \
    template int batched_occupancy_t<F>();                                                    \
    template cudaError_t launch_multi_t<F>(int, const StepArgs&, int, cudaStream_t, bool);    \
    template int multi_occupancy_t<F>(int);                                                   \
    template int step_occupancy_t<F>(int, int);                                               \
    template bool has_tma_t<F>();                                                             \
    template bool has_async_t<F>();                                                           \
    template bool has_pairs_t<F>();                                                           \
    template cudaError_t launch_init_t<F>(const StepArgs&, const double*, int, int,           \
                                          cudaStream_t);                                      \
    template cudaError_t launch_fields_t<F>(const AuxArgs&, int, cudaStream_t);               \
    template cudaError_t launch_diag_t<F>(const AuxArgs&, int, cudaStream_t);                 \
    template cudaError_t launch_populations_t<F>(const AuxArgs&, int, double*, double*,       \
                                                 cudaStream_t);

}  // namespace lbm
