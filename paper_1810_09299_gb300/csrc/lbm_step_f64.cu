// lbm_step_f64.cu -- instantiation of the step, field, init and state kernels
// for the CodecF64 storage codec (see lbm_device.cuh).
#include "lbm_kernels.cuh"

AXILBM_INSTANTIATE(f64, axilbm::CodecF64)
