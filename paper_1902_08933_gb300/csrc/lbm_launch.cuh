// lbm_launch.cuh -- host-side launchers of the kernels of one storage form.
// Included by lbm_form<N>.cu, which instantiates them for its form.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

template <int FORM, int TX>
static cudaError_t launch_step_tx(const StepArgs& a, int nwork, cudaStream_t s) {
    const size_t smem = StepSmem<FORM, TX>::bytes;
    step_kernel<FORM, TX><<<nwork, TX, smem, s>>>(a);
    return cudaGetLastError();
}

template <int FORM>
cudaError_t launch_step_t(int tile_x, const StepArgs& a, int nwork, cudaStream_t s) {
    if (nwork <= 0) return cudaSuccess;
    switch (tile_x) {
        case 32: return launch_step_tx<FORM, 32>(a, nwork, s);
        case 64: return launch_step_tx<FORM, 64>(a, nwork, s);
        case 128: return launch_step_tx<FORM, 128>(a, nwork, s);
        case 256: return launch_step_tx<FORM, 256>(a, nwork, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int FORM, int TX>
static cudaError_t prep_tx() {
    return cudaFuncSetAttribute(step_kernel<FORM, TX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)StepSmem<FORM, TX>::bytes);
}

template <int FORM>
cudaError_t prepare_step_t() {
    cudaError_t e;
    if ((e = prep_tx<FORM, 32>()) != cudaSuccess) return e;
    if ((e = prep_tx<FORM, 64>()) != cudaSuccess) return e;
    if ((e = prep_tx<FORM, 128>()) != cudaSuccess) return e;
    return prep_tx<FORM, 256>();
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

template <int FORM>
int step_occupancy_t(int tile_x) {
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (tile_x) {
        case 32: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel<FORM, 32>, 32, StepSmem<FORM, 32>::bytes); break;
        case 64: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel<FORM, 64>, 64, StepSmem<FORM, 64>::bytes); break;
        case 128: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel<FORM, 128>, 128, StepSmem<FORM, 128>::bytes); break;
        case 256: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel<FORM, 256>, 256, StepSmem<FORM, 256>::bytes); break;
        default: break;
    }
    return e == cudaSuccess ? n : 0;
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
    diag_final<<<1, 32, 0, s>>>(a.partials, kDiagBlocks, a.result);
    return cudaGetLastError();
}

template <int FORM>
cudaError_t launch_populations_t(const AuxArgs& a, int ncells, double* out_h, double* out_g,
                                 cudaStream_t s) {
    populations_pass<FORM><<<grid_for(ncells, 256), 256, 0, s>>>(a, out_h, out_g);
    return cudaGetLastError();
}

#define LBM_INSTANTIATE_FORM(F)                                                               \
    template cudaError_t launch_step_t<F>(int, const StepArgs&, int, cudaStream_t);           \
    template cudaError_t prepare_step_t<F>();                                                 \
    template size_t step_smem_t<F>(int);                                                      \
    template int step_occupancy_t<F>(int);                                                    \
    template cudaError_t launch_init_t<F>(const StepArgs&, const double*, int, int,           \
                                          cudaStream_t);                                      \
    template cudaError_t launch_fields_t<F>(const AuxArgs&, int, cudaStream_t);               \
    template cudaError_t launch_diag_t<F>(const AuxArgs&, int, cudaStream_t);                 \
    template cudaError_t launch_populations_t<F>(const AuxArgs&, int, double*, double*,       \
                                                 cudaStream_t);

}  // namespace lbm
