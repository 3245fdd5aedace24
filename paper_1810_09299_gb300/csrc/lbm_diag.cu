// lbm_diag.cu -- FP64 diagnostics of one case (compensated, deterministic
// reductions) and the initial phase-field shapes of the paper's tests (Sec. 3).
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>

#include "../../include/lbm.h"
#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace axilbm {

namespace {

constexpr int kDiagBlocks = kDiagPartials / 18;  // 2 x 152 SMs; fixed so the summation order is fixed
constexpr int kDiagThreads = 256;

// Neumaier compensated accumulation.
struct KSum {
    double s, c;
    __device__ void add(double x) {
        const double t = s + x;
        if (fabs(s) >= fabs(x)) c += (s - t) + x;
        else c += (x - t) + s;
        s = t;
    }
    __device__ void merge(const KSum& o) {
        add(o.s);
        c += o.c;
    }
    __device__ double value() const { return s + c; }
};

// Quantities: 0 mass, 1 kinetic, 2 z-moment, 3 p in liquid, 4 weight in liquid,
// 5 p in gas, 6 weight in gas (sums); 7 umax, 8 phi_min, 9 phi_max (extrema);
// 10 non-finite count (sum).
__global__ void __launch_bounds__(kDiagThreads) diag_partial_kernel(const double* __restrict__ F, int nz, int nr,
                                                                    double* __restrict__ partials) {
    const int64_t n = (int64_t)nz * nr;
    KSum acc[7] = {};
    double umax = 0.0, pmin = INFINITY, pmax = -INFINITY, bad = 0.0;
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(o / nr), j = (int)(o - (int64_t)k * nr);
        const double r = j + 0.5, z = k + 0.5;
        const double phi = F[o], rho = F[n + o], uz = F[2 * n + o], ur = F[3 * n + o], p = F[4 * n + o];
        if (!isfinite(phi) || !isfinite(uz) || !isfinite(ur) || !isfinite(p)) {
            bad += 1.0;
            continue;
        }
        const double uu = uz * uz + ur * ur;
        acc[0].add(r * phi);
        acc[1].add(0.5 * r * rho * uu);
        acc[2].add(r * z * phi);
        if (phi > 0.99) {
            acc[3].add(r * p);
            acc[4].add(r);
        }
        if (phi < 0.01) {
            acc[5].add(r * p);
            acc[6].add(r);
        }
        umax = fmax(umax, sqrt(uu));
        pmin = fmin(pmin, phi);
        pmax = fmax(pmax, phi);
    }
    __shared__ double sh[kDiagThreads][2 * 7 + 4];
    for (int q = 0; q < 7; ++q) {
        sh[threadIdx.x][2 * q] = acc[q].s;
        sh[threadIdx.x][2 * q + 1] = acc[q].c;
    }
    sh[threadIdx.x][14] = umax;
    sh[threadIdx.x][15] = pmin;
    sh[threadIdx.x][16] = pmax;
    sh[threadIdx.x][17] = bad;
    __syncthreads();
    for (int stride = kDiagThreads / 2; stride > 0; stride >>= 1) {
        if (threadIdx.x < stride) {
            double* a = sh[threadIdx.x];
            const double* b = sh[threadIdx.x + stride];
            for (int q = 0; q < 7; ++q) {
                KSum x{a[2 * q], a[2 * q + 1]};
                x.merge(KSum{b[2 * q], b[2 * q + 1]});
                a[2 * q] = x.s;
                a[2 * q + 1] = x.c;
            }
            a[14] = fmax(a[14], b[14]);
            a[15] = fmin(a[15], b[15]);
            a[16] = fmax(a[16], b[16]);
            a[17] += b[17];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int q = 0; q < 18; ++q) partials[blockIdx.x * 18 + q] = sh[0][q];
    }
}

// One partial record: 7 compensated sums, 3 extrema, the non-finite count.
__device__ __forceinline__ void merge_partial(double* a, const double* b) {
    for (int q = 0; q < 7; ++q) {
        KSum x{a[2 * q], a[2 * q + 1]};
        x.merge(KSum{b[2 * q], b[2 * q + 1]});
        a[2 * q] = x.s;
        a[2 * q + 1] = x.c;
    }
    a[14] = fmax(a[14], b[14]);
    a[15] = fmin(a[15], b[15]);
    a[16] = fmax(a[16], b[16]);
    a[17] += b[17];
}

// Contribution of the axis link (k, k+1) to the length of the phi > 1/2 set on
// the axis row (linear crossing); the last link wraps when z is periodic and
// is half a cell at a wall.
__device__ __forceinline__ double axis_link(const double* __restrict__ F, int k, int nz, int nr, int zper) {
    const double a = F[(int64_t)k * nr] - 0.5;
    int kn = k + 1;
    if (kn >= nz) {
        if (!zper) return a > 0 ? 0.5 : 0.0;
        kn = 0;
    }
    const double b = F[(int64_t)kn * nr] - 0.5;
    if (a > 0 && b > 0) return 1.0;
    if (a > 0 && b <= 0) return a / (a - b);
    if (a <= 0 && b > 0) return b / (b - a);
    return 0.0;
}

// Final combination and the interface lengths, one block of kFinalThreads.
// Every sum runs in a fixed order (fixed-shape trees), so the result is
// deterministic.
constexpr int kFinalThreads = 256;
static_assert(kDiagBlocks <= 2 * kFinalThreads, "one fold into the first kFinalThreads partials");
__global__ void __launch_bounds__(kFinalThreads) diag_final_kernel(const double* __restrict__ F, int nz, int nr,
                                                                   int zper, double step,
                                                                   const double* __restrict__ partials,
                                                                   double* __restrict__ out) {
    __shared__ double sp[kDiagBlocks][18];
    __shared__ double slen[kFinalThreads];
    __shared__ int sjmin;
    const int t = threadIdx.x;
    for (int i = t; i < kDiagBlocks * 18; i += kFinalThreads) (&sp[0][0])[i] = partials[i];
    if (t == 0) sjmin = nr;
    __syncthreads();
    // partial records: fold kDiagBlocks into kFinalThreads, then a halving tree
    if (t + kFinalThreads < kDiagBlocks) merge_partial(sp[t], sp[t + kFinalThreads]);
    __syncthreads();
    for (int stride = kFinalThreads / 2; stride > 0; stride >>= 1) {
        if (t < stride) merge_partial(sp[t], sp[t + stride]);
        __syncthreads();
    }
    // axis half-length: per-thread sums over k = t, t + T, ... then a halving tree
    double len = 0.0;
    for (int k = t; k < nz; k += kFinalThreads) len += axis_link(F, k, nz, nr, zper);
    slen[t] = len;
    __syncthreads();
    for (int stride = kFinalThreads / 2; stride > 0; stride >>= 1) {
        if (t < stride) slen[t] += slen[t + stride];
        __syncthreads();
    }
    const double mass = KSum{sp[0][0], sp[0][1]}.value();
    const double zc = KSum{sp[0][4], sp[0][5]}.value() / mass;
    // radial crossing on the row nearest the centroid: the first outward crossing
    int kc = (int)floor(zc);
    kc = kc < 0 ? 0 : (kc >= nz ? nz - 1 : kc);
    for (int j = t; j + 1 < nr; j += kFinalThreads) {
        const double a = F[(int64_t)kc * nr + j] - 0.5, b = F[(int64_t)kc * nr + j + 1] - 0.5;
        if (a > 0 && b <= 0) {
            atomicMin(&sjmin, j);
            break;
        }
    }
    __syncthreads();
    if (t != 0) return;
    double rc = 0.0;
    if (sjmin + 1 < nr) {
        const double a = F[(int64_t)kc * nr + sjmin] - 0.5, b = F[(int64_t)kc * nr + sjmin + 1] - 0.5;
        rc = (sjmin + 0.5) + a / (a - b);
    }
    double axis = slen[0];
    if (!zper && F[0] - 0.5 > 0) axis += 0.5;
    const double win = KSum{sp[0][8], sp[0][9]}.value(), wout = KSum{sp[0][12], sp[0][13]}.value();
    const double dp = (win > 0 ? KSum{sp[0][6], sp[0][7]}.value() / win : 0.0) -
                      (wout > 0 ? KSum{sp[0][10], sp[0][11]}.value() / wout : 0.0);
    out[0] = step;
    out[1] = mass;
    out[2] = KSum{sp[0][2], sp[0][3]}.value();
    out[3] = zc;
    out[4] = dp;
    out[5] = sp[0][14];
    out[6] = sp[0][15];
    out[7] = sp[0][16];
    out[8] = 0.5 * axis;
    out[9] = rc;
    out[10] = sp[0][17];
}

// ---------------------------------------------------------------- shapes
struct ShapeArgs {
    double a[8];
};

__global__ void shape_kernel(int shape, ShapeArgs A, int nz, int nr, double* __restrict__ phi) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
    if (j >= nr || k >= nz) return;
    const double z = k + 0.5, r = j + 0.5;
    double v = 0.0;
    switch (shape) {
        case 0: {  // flat: {z_i, W, axis}
            const double x = (A.a[2] == 0.0) ? z : r;
            v = 0.5 + 0.5 * tanh(2.0 * (A.a[0] - x) / A.a[1]);
            break;
        }
        case 1:
        case 5: {  // sphere / bubble: {z_c, R, W}
            const double d = sqrt((z - A.a[0]) * (z - A.a[0]) + r * r);
            v = 0.5 + 0.5 * tanh(2.0 * (A.a[1] - d) / A.a[2]);
            if (shape == 5) v = 1.0 - v;
            break;
        }
        case 2: {  // ellipsoid: {z_c, R_z, R_r, W}
            const double Re = cbrt(A.a[2] * A.a[2] * A.a[1]);
            const double q = sqrt((z - A.a[0]) * (z - A.a[0]) / (A.a[1] * A.a[1]) + r * r / (A.a[2] * A.a[2]));
            v = 0.5 + 0.5 * tanh(2.0 * Re * (1.0 - q) / A.a[3]);
            break;
        }
        case 3: {  // P2 drop: {z_c, R0, eps, W}
            const double d = sqrt((z - A.a[0]) * (z - A.a[0]) + r * r);
            const double c = (z - A.a[0]) / fmax(d, 1e-300);
            const double Rs = A.a[1] * (1.0 + A.a[2] * 0.5 * (3.0 * c * c - 1.0));
            v = 0.5 + 0.5 * tanh(2.0 * (Rs - d) / A.a[3]);
            break;
        }
        case 4: {  // thread: {R, amp, lambda, theta, W}
            const double d = A.a[1] * cos(2.0 * M_PI * z / A.a[2] + A.a[3]);
            v = 0.5 + 0.5 * tanh(2.0 * (A.a[0] + d - r) / A.a[4]);
            break;
        }
        default:
            v = 0.0;
    }
    phi[(int64_t)k * nr + j] = v;
}

}  // namespace

int diag_partials_size() { return kDiagPartials; }

cudaError_t launch_diag(const double* fields, int nz, int nr, int zper, double step, double* partials, double* out,
                        cudaStream_t st) {
    diag_partial_kernel<<<kDiagBlocks, kDiagThreads, 0, st>>>(fields, nz, nr, partials);
    diag_final_kernel<<<1, kFinalThreads, 0, st>>>(fields, nz, nr, zper, step, partials, out);
    return cudaGetLastError();
}

cudaError_t launch_shape(int shape, const double* args, int nargs, int nz, int nr, double* phi0, cudaStream_t st) {
    ShapeArgs A{};
    for (int i = 0; i < nargs && i < 8; ++i) A.a[i] = args[i];
    dim3 grid((nr + 127) / 128, nz);
    shape_kernel<<<grid, 128, 0, st>>>(shape, A, nz, nr, phi0);
    return cudaGetLastError();
}

}  // namespace axilbm

// ---------------------------------------------------------------- bounded-wait self-test
namespace {
// An mbarrier expecting two arrivals gets one, so its phase never completes:
// the bounded wait must give up after `tries` polls and raise the status word.
__global__ void selftest_wait_kernel(int tries, int* status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) axilbm::mbar_init(&bar, 2);
    __syncthreads();
    if (threadIdx.x == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(axilbm::smem_addr(&bar)) : "memory");
    axilbm::mbar_wait_bounded(&bar, 0, status, tries);
}
}  // namespace

extern "C" int lbm_selftest_bounded_wait(int32_t tries, void* stream, int32_t* device_status_word) {
    if (tries < 1 || !device_status_word) return LBM_ERR_INVALID_ARG;
    selftest_wait_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(tries, device_status_word);
    if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
    int st = 0;
    if (cudaMemcpyAsync(&st, device_status_word, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream) !=
            cudaSuccess ||
        cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    return st != 0 ? LBM_ERR_TIMEOUT : LBM_OK;
}

// ---------------------------------------------------------------- allocation-free reduction
// lbm_diag_reduce_noalloc: the diagnostics reduction for callers that cannot
// allocate device memory when they need the numbers (for example a caller
// whose device memory is entirely held by its own pool, or a monitoring loop
// that must not pay for an allocation).  Its only scratch, the per-block
// partial sums, is a fixed static device array of this module.
namespace {

constexpr int kScratchDoubles = axilbm::kDiagPartials;  // 304 blocks x 18 doubles = 43,776 bytes
constexpr int64_t kNoAllocMaxNodes = 2147483647;       // nz * nr must fit a signed 32-bit count
constexpr int kMaxDevices = 64;

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) double g_diag_scratch[kScratchDoubles];

std::mutex g_scratch_mutex;
double* g_scratch_addr[kMaxDevices] = {};  // device address of g_diag_scratch, per device

}  // namespace

extern "C" int lbm_diag_reduce_noalloc(const double* d_fields, int32_t nz, int32_t nr, int32_t z_periodic,
                                       double step, double* d_out, void* stream) {
    if (!d_fields || !d_out || nz < 1 || nr < 1 || (z_periodic != 0 && z_periodic != 1))
        return LBM_ERR_INVALID_ARG;
    if ((int64_t)nz * nr > kNoAllocMaxNodes) return LBM_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return LBM_ERR_INVALID_ARG;
    double* scratch = nullptr;
    {
        // one-time set-up on this device (current device): the host-side name
        // g_diag_scratch is not a device address, so look the address up
        std::lock_guard<std::mutex> lock(g_scratch_mutex);
        if (!g_scratch_addr[dev]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_diag_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return LBM_ERR_CUDA;
            }
            g_scratch_addr[dev] = (double*)p;
        }
        scratch = g_scratch_addr[dev];
    }
    // Every partial slot is overwritten by the first kernel before the second
    // reads it, so nothing from an earlier call needs clearing.
    cudaError_t e = axilbm::launch_diag(d_fields, nz, nr, z_periodic, step, scratch, d_out, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    return LBM_OK;
}
