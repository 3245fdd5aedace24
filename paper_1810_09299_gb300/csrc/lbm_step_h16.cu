// lbm_step_h16.cu -- instantiation of the step, field, init and state kernels
// for the CodecH16 storage codec (see lbm_device.cuh).
#include "lbm_kernels.cuh"

AXILBM_INSTANTIATE(h16, axilbm::CodecH16)
