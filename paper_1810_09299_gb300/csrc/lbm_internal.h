// lbm_internal.h -- host-side declarations shared by the C ABI and the
// per-precision kernel translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace axilbm {

struct CaseDev;
struct TileDev;

// Bytes of one storage block (the stored values of 32 nodes: f_0, f_1..8,
// g_0..8, chi_z, chi_r, p), padded to a multiple of 128 bytes; the element
// sizes are those of f_0, of a population and of the arithmetic type.
constexpr int block_bytes_of(int f0_size, int pt_size, int real_size) {
    return (32 * f0_size + 17 * 32 * pt_size + 3 * 32 * real_size + 127) / 128 * 128;
}

// Rate modes of the step kernels: general rates read from the case record, or
// a rate pattern every case of the handle shares and the kernels know at
// compile time -- the paper's (Sec. 3.1: S^f = diag(1, 1, 1, s, s, s, s, 1, 1),
// S^g = 1 except s_1 = s_7 = s_8 = 1/tau_g) or the same choice for the
// raw-moment collision (f: s on raw moments 1, 2, 6, 7; g: 1/tau_g on 3, 4, 5).
constexpr int kRatesGeneral = 0, kRatesPaper = 1, kRatesPaperRaw = 2;

// Device buffers of a handle: two arrays of `total / 32` blocks (one block per
// 32 nodes, see Block in lbm_device.cuh); index [parity] selects the buffer
// read by the next step.
struct DeviceState {
    void* blk[2];
    void* cases;  // CaseDev[ncases] on the device
    int64_t total;
    int rate_mode;     // kRatesGeneral, or the rate pattern every case shares (see below)
    const void* tmaps;  // CUtensorMap[ncases][2 tile heights][kMapsPerCase] in device memory
    int* status;        // device status word: nonzero after a bounded wait gave up
};

#define AXILBM_DECLARE(NAME)                                                                                       \
    cudaError_t launch_step_##NAME(const DeviceState& D, int parity, int variant, const TileDev* tiles, int ntiles, \
                                   cudaStream_t st);                                                               \
    cudaError_t launch_fields_##NAME(const DeviceState& D, int parity, const TileDev* tiles, int ntiles,            \
                                     double* out, cudaStream_t st);                                                \
    cudaError_t launch_init_##NAME(const DeviceState& D, int parity, const TileDev* tiles8, int ntiles,             \
                                   const double* phi0, int64_t base, cudaStream_t st);                             \
    cudaError_t launch_get_state_##NAME(const DeviceState& D, int parity, const CaseDev& C, double* f, double* g,   \
                                        double* aux, cudaStream_t st);                                             \
    cudaError_t launch_set_state_##NAME(const DeviceState& D, int parity, const CaseDev& C, const double* f,        \
                                        const double* g, const double* aux, cudaStream_t st);

AXILBM_DECLARE(f64)
AXILBM_DECLARE(f32)
AXILBM_DECLARE(h16)
AXILBM_DECLARE(b16)
#undef AXILBM_DECLARE

constexpr int kNumVariants = 8;
// tile height along z of each step-kernel variant (tile width is one warp along r);
// variants 3 and 4 stage the tile through shared memory with TMA tensor loads;
// variants 5 and 6 update two nodes of a column per thread, one after the
// other (CTAs of 8 warps; 6 parks the second node's inputs in shared memory
// while the first is updated), in FP32 arithmetic, and run the one-node
// kernel of their tile height in FP64; variant 7 updates the two nodes
// together in packed FP32x2 lanes (FP16 storage; the other precisions run
// variant 5's kernel there)
constexpr int kVariantTZ[kNumVariants] = {8, 16, 4, 8, 16, 16, 16, 16};
constexpr bool kVariantTMA[kNumVariants] = {false, false, false, true, true, false, false, false};
// tensor maps per case and tile height: the case's blocks in buffer 0 and 1
// with a box of the tile's rows plus two above and below (staging, [0], [1]),
// and with a box of the tile's rows only (L2 prefetch, [2], [3])
constexpr int kMapsPerCase = 4;

// Diagnostics (lbm_diag.cu): reduce dense FP64 fields of one case into a
// 11-double record; `partials` is scratch of at least diag_partials_size()
// doubles.  Deterministic (fixed block count and order).
constexpr int kDiagPartials = 304 * 18;  // 304 blocks x 18 doubles
int diag_partials_size();
cudaError_t launch_diag(const double* fields, int nz, int nr, int zper, double step, double* partials,
                        double* out, cudaStream_t st);

// Drops on the axis row (lbm_diag.cu): out[3 + 4 * kMaxAxisDrops] doubles,
// rows: nz doubles of scratch.
constexpr int kMaxAxisDrops = 64;
cudaError_t launch_axis_drops(const double* fields, int nz, int nr, int zper, int max_drops, double* rows, double* out,
                              cudaStream_t st);

// Initial shapes (lbm_diag.cu): phi0 [nz][nr] on the device.
cudaError_t launch_shape(int shape, const double* args, int nargs, int nz, int nr, double* phi0, cudaStream_t st);

}  // namespace axilbm
