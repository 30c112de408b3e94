// Kernels and launchers of storage form 5 (see the form table in lbm_device.cuh).
#include "lbm_launch.cuh"
namespace lbm {
LBM_INSTANTIATE_FORM(5)
}
