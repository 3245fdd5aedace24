// lbm_step_f32.cu -- instantiation of the step, field, init and state kernels
// for the CodecF32 storage codec (see lbm_device.cuh).
#include "lbm_kernels.cuh"

AXILBM_INSTANTIATE(f32, axilbm::CodecF32)
