// lbm_step_b16.cu -- instantiation of the step, field, init and state kernels
// for the CodecB16 storage codec (see lbm_device.cuh).
#include "lbm_kernels.cuh"

AXILBM_INSTANTIATE(b16, axilbm::CodecB16)
