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
// 5 p in gas, 6 weight in gas (sums); 7 max |u|^2, 8 phi_min, 9 phi_max
// (extrema); 10 non-finite count (sum).  A partial record is 18 doubles:
// (sum, compensation) of quantities 0-6, then 7-10.
constexpr int kSums = 7;

// A compensated pair (s, c) from lane + off of the warp (a shuffle of both).
__device__ __forceinline__ KSum shfl_down_ksum(const KSum& x, int off) {
    return KSum{__shfl_down_sync(0xffffffffu, x.s, off), __shfl_down_sync(0xffffffffu, x.c, off)};
}

// Combine the compensated pairs (v, vc)[0 .. count) held in shared memory with
// stride `stride` (one per partial record) into lane 0 of the calling warp:
// each lane merges its share in a fixed order, then a fixed shuffle tree
// merges the lanes.  Every sum is compensated (Neumaier).
__device__ __forceinline__ KSum warp_ksum(const double* v, const double* vc, int count, int stride) {
    const int lane = threadIdx.x & 31;
    KSum acc{0.0, 0.0};
    for (int i = lane; i < count; i += 32) acc.merge(KSum{v[(size_t)i * stride], vc[(size_t)i * stride]});
    for (int off = 16; off > 0; off >>= 1) {
        const KSum o = shfl_down_ksum(acc, off);
        if (lane + off < 32) acc.merge(o);
    }
    return acc;
}

// The plain sum of v[0 .. count) (stride as above) into lane 0: each lane adds
// its share in a fixed order, then a fixed pairwise shuffle tree.  Used inside
// a block, where a thread holds few nodes: pairwise summation of the block's
// values keeps the error near log2(values) rounding units.
__device__ __forceinline__ double warp_sum(const double* v, int count, int stride) {
    const int lane = threadIdx.x & 31;
    double acc = 0.0;
    for (int i = lane; i < count; i += 32) acc += v[(size_t)i * stride];
    for (int off = 16; off > 0; off >>= 1) {
        const double o = __shfl_down_sync(0xffffffffu, acc, off);
        if (lane + off < 32) acc += o;
    }
    return acc;
}

// The extrema and the count the same way: max |u|^2, min phi, max phi, count.
__device__ __forceinline__ void warp_extrema(const double* uu, const double* lo, const double* hi,
                                             const double* bad, int count, int stride, double out[4]) {
    const int lane = threadIdx.x & 31;
    double m = 0.0, mn = INFINITY, mx = -INFINITY, nb = 0.0;
    for (int i = lane; i < count; i += 32) {
        m = fmax(m, uu[(size_t)i * stride]);
        mn = fmin(mn, lo[(size_t)i * stride]);
        mx = fmax(mx, hi[(size_t)i * stride]);
        nb += bad[(size_t)i * stride];
    }
    for (int off = 16; off > 0; off >>= 1) {
        m = fmax(m, __shfl_down_sync(0xffffffffu, m, off));
        mn = fmin(mn, __shfl_down_sync(0xffffffffu, mn, off));
        mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, off));
        const double o = __shfl_down_sync(0xffffffffu, nb, off);
        if (lane + off < 32) nb += o;
    }
    out[0] = m;
    out[1] = mn;
    out[2] = mx;
    out[3] = nb;
}

// One partial record per block.  Rows k = blockIdx.x, blockIdx.x + gridDim.x,
// ...; within a row each thread takes the columns j = threadIdx.x + 256 i, so a
// thread holds only a few nodes and sums them plainly; the block's 256 values
// of each quantity are then summed pairwise by one warp per quantity (warps
// 0-6 the sums, warp 7 the extrema and the count).  The records of the blocks
// are combined with compensated sums by diag_final_kernel.
__global__ void __launch_bounds__(kDiagThreads) diag_partial_kernel(const double* __restrict__ F, int nz, int nr,
                                                                    double* __restrict__ partials) {
    static_assert(kDiagThreads == 32 * (kSums + 1), "one warp per sum plus one");
    const int64_t n = (int64_t)nz * nr;
    double acc[kSums] = {};
    double uu_max = 0.0, pmin = INFINITY, pmax = -INFINITY, bad = 0.0;
    for (int k = blockIdx.x; k < nz; k += gridDim.x) {
        const double z = k + 0.5;
        for (int j = threadIdx.x; j < nr; j += blockDim.x) {
            const int64_t o = (int64_t)k * nr + j;
            const double r = j + 0.5;
            const double phi = F[o], rho = F[n + o], uz = F[2 * n + o], ur = F[3 * n + o], p = F[4 * n + o];
            if (!isfinite(phi) || !isfinite(uz) || !isfinite(ur) || !isfinite(p)) {
                bad += 1.0;
                continue;
            }
            const double uu = uz * uz + ur * ur;
            acc[0] += r * phi;
            acc[1] += 0.5 * r * rho * uu;
            acc[2] += r * z * phi;
            if (phi > 0.99) {
                acc[3] += r * p;
                acc[4] += r;
            }
            if (phi < 0.01) {
                acc[5] += r * p;
                acc[6] += r;
            }
            uu_max = fmax(uu_max, uu);
            pmin = fmin(pmin, phi);
            pmax = fmax(pmax, phi);
        }
    }
    __shared__ double sh[kSums + 4][kDiagThreads];
    for (int q = 0; q < kSums; ++q) sh[q][threadIdx.x] = acc[q];
    sh[kSums][threadIdx.x] = uu_max;
    sh[kSums + 1][threadIdx.x] = pmin;
    sh[kSums + 2][threadIdx.x] = pmax;
    sh[kSums + 3][threadIdx.x] = bad;
    __syncthreads();
    const int w = threadIdx.x >> 5;
    double* out = partials + (size_t)blockIdx.x * 18;
    if (w < kSums) {
        const double t = warp_sum(sh[w], kDiagThreads, 1);
        if ((threadIdx.x & 31) == 0) {
            out[2 * w] = t;
            out[2 * w + 1] = 0.0;
        }
    } else {
        double e[4];
        warp_extrema(sh[kSums], sh[kSums + 1], sh[kSums + 2], sh[kSums + 3], kDiagThreads, 1, e);
        if ((threadIdx.x & 31) == 0)
            for (int q = 0; q < 4; ++q) out[14 + q] = e[q];
    }
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

// Final combination and the interface lengths, one block of kFinalThreads:
// warps 0-6 combine one sum each over the partial records and warp 7 the
// extrema and the count, every one in a fixed order (compensated sums), so
// the result is deterministic.
constexpr int kFinalThreads = 256;
static_assert(kFinalThreads == 32 * (kSums + 1), "one warp per sum plus one");
__global__ void __launch_bounds__(kFinalThreads) diag_final_kernel(const double* __restrict__ F, int nz, int nr,
                                                                   int zper, double step,
                                                                   const double* __restrict__ partials,
                                                                   double* __restrict__ out) {
    __shared__ double sp[kDiagBlocks][18];
    __shared__ double sres[18];
    __shared__ double slen[kFinalThreads];
    __shared__ int sjmin;
    const int t = threadIdx.x;
    for (int i = t; i < kDiagBlocks * 18; i += kFinalThreads) (&sp[0][0])[i] = partials[i];
    if (t == 0) sjmin = nr;
    __syncthreads();
    const int w = t >> 5;
    if (w < kSums) {
        const KSum r = warp_ksum(&sp[0][2 * w], &sp[0][2 * w + 1], kDiagBlocks, 18);
        if ((t & 31) == 0) {
            sres[2 * w] = r.s;
            sres[2 * w + 1] = r.c;
        }
    } else {
        double e[4];
        warp_extrema(&sp[0][14], &sp[0][15], &sp[0][16], &sp[0][17], kDiagBlocks, 18, e);
        if ((t & 31) == 0)
            for (int q = 0; q < 4; ++q) sres[14 + q] = e[q];
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
    __syncthreads();
    const double mass = KSum{sres[0], sres[1]}.value();
    const double zc = KSum{sres[4], sres[5]}.value() / mass;
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
    const double win = KSum{sres[8], sres[9]}.value(), wout = KSum{sres[12], sres[13]}.value();
    const double dp = (win > 0 ? KSum{sres[6], sres[7]}.value() / win : 0.0) -
                      (wout > 0 ? KSum{sres[10], sres[11]}.value() / wout : 0.0);
    out[0] = step;
    out[1] = mass;
    out[2] = KSum{sres[2], sres[3]}.value();
    out[3] = zc;
    out[4] = dp;
    out[5] = sqrt(sres[14]);  // |u|max from the largest |u|^2
    out[6] = sres[15];
    out[7] = sres[16];
    out[8] = 0.5 * axis;
    out[9] = rc;
    out[10] = sres[17];
}

// ---------------------------------------------------------------- drops on the axis
// The liquid bodies a breaking thread forms (Sec. 3.3), read off the axis row
// j = 0: every maximal run of axis nodes with phi > 1/2 is one drop.  The rows
// of the case are split between the drops at one row inside each gas gap (the
// row of least r-weighted phi of the gap, first on ties), so every row belongs
// to exactly one drop and a drop's volume is 2 pi sum r phi over its rows.
// Its ends are the linearly interpolated phi = 1/2 crossings on the axis (a
// wall plane where the run reaches a z wall).  In a periodic case the rows
// wrap; with no gap at all the whole axis is one unbroken body.
//
// Output (FP64): out[0] = number of drops, out[1] = min phi on the axis row,
// out[2] = row of that minimum + 1/2 (its z), then for each of the first
// min(number, max_drops) drops in z order (z_start, z_end, volume, radius of
// the sphere of that volume); z_end < z_start for a drop that wraps a periodic
// boundary.  rows: scratch of nz doubles.
constexpr int kAxisThreads = 256;

__device__ __forceinline__ double axis_phi(const double* F, int nr, int k) { return F[(int64_t)k * nr]; }

// z of the phi = 1/2 crossing between axis rows k and k + 1 (k + 1 taken
// modulo nz, positions unwrapped: z may exceed nz by less than one row).
__device__ __forceinline__ double axis_crossing(const double* F, int nz, int nr, int k) {
    const double a = axis_phi(F, nr, k), b = axis_phi(F, nr, (k + 1) % nz);
    return (k + 0.5) + (0.5 - a) / (b - a);
}

__global__ void __launch_bounds__(kAxisThreads) axis_drops_kernel(const double* __restrict__ F, int nz, int nr,
                                                                  int zper, int max_drops,
                                                                  double* __restrict__ rows,
                                                                  double* __restrict__ out) {
    for (int k = threadIdx.x; k < nz; k += blockDim.x) {
        double s = 0.0;
        // separately rounded products and sums in r order (no contraction)
        for (int j = 0; j < nr; ++j) s = __dadd_rn(s, __dmul_rn(j + 0.5, F[(int64_t)k * nr + j]));
        rows[k] = s;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const double two_pi = 6.283185307179586;
    double pmin = INFINITY;
    int kmin = 0;
    int start = -1;  // a gas row of the axis to start the scan at (periodic)
    for (int k = 0; k < nz; ++k) {
        const double v = axis_phi(F, nr, k);
        if (v < pmin) {
            pmin = v;
            kmin = k;
        }
        if (start < 0 && !(v > 0.5)) start = k;
    }
    out[1] = pmin;
    out[2] = kmin + 0.5;
    const auto put = [&](int drop, int field, double v) {
        if (drop < max_drops) out[3 + 4 * drop + field] = v;
    };
    const auto close_drop = [&](int drop, double v) {
        put(drop, 2, two_pi * v);
        put(drop, 3, cbrt(3.0 * two_pi * v / (4.0 * M_PI)));
    };
    if (start < 0) {  // liquid along the whole axis: one unbroken body
        double vol = 0.0;
        for (int k = 0; k < nz; ++k) vol += rows[k];
        out[0] = 1.0;
        put(0, 0, 0.0);
        put(0, 1, (double)nz);
        close_drop(0, vol);
        return;
    }
    if (zper) {
        // start the scan at the first row of a gas gap, so that the rows
        // before it (cyclically) end the last drop
        int n = 0;
        while (n < nz && !(axis_phi(F, nr, (start + nz - 1) % nz) > 0.5)) {
            start = (start + nz - 1) % nz;
            ++n;
        }
        if (n == nz) {  // gas along the whole axis: no drop
            out[0] = 0.0;
            return;
        }
    } else {
        start = 0;
    }
    // One pass over the rows in scan order.  Inside a gap the rows before its
    // lightest row go to the drop before the gap, the rest to the drop after it.
    int ndrops = 0;
    double vol = 0.0;                      // rows of the current drop so far
    double gap_before = 0.0, gap_after = 0.0, gap_min = 0.0;
    double lead_before = 0.0;              // periodic: first gap's share of the last drop
    bool in_gap = false, first_row = true;
    for (int i = 0; i < nz; ++i) {
        const int k = zper ? (start + i) % nz : i;
        const int kp = (k + nz - 1) % nz;  // the row before k (cyclically)
        const bool liquid = axis_phi(F, nr, k) > 0.5;
        if (!liquid) {
            if (!in_gap) {
                // a gap opens: the drop before it (if any) ends before this row
                if (!first_row) {
                    double ze = axis_crossing(F, nz, nr, kp);
                    if (ze >= nz) ze -= nz;
                    put(ndrops - 1, 1, ze);
                }
                in_gap = true;
                gap_before = 0.0;
                gap_after = rows[k];
                gap_min = rows[k];
            } else if (rows[k] < gap_min) {
                gap_before += gap_after;
                gap_after = rows[k];
                gap_min = rows[k];
            } else {
                gap_after += rows[k];
            }
        } else {
            if (in_gap || first_row) {
                // a drop starts at this row
                if (ndrops > 0) {
                    close_drop(ndrops - 1, vol + gap_before);
                    vol = gap_after;
                } else {
                    // the first drop: a leading gap of a walled case is all its;
                    // in a periodic case the part before the cut wraps to the last drop
                    if (zper) {
                        lead_before = gap_before;
                        vol = gap_after;
                    } else {
                        vol = gap_before + gap_after;
                    }
                }
                double zs = 0.0;  // a drop touching the wall z = 0 starts at the wall plane
                if (!(first_row && !zper)) {
                    zs = axis_crossing(F, nz, nr, kp);
                    if (zs >= nz) zs -= nz;
                }
                put(ndrops, 0, zs);
                ++ndrops;
                in_gap = false;
                gap_before = gap_after = 0.0;
            }
            vol += rows[k];
        }
        first_row = false;
    }
    if (ndrops > 0) {
        if (zper) {
            // the scan started at a gap's first row, so it ends inside the last drop
            double ze = axis_crossing(F, nz, nr, (start + nz - 1) % nz);
            if (ze >= nz) ze -= nz;
            put(ndrops - 1, 1, ze);
            close_drop(ndrops - 1, vol + lead_before);
        } else if (in_gap) {
            close_drop(ndrops - 1, vol + gap_before + gap_after);
        } else {
            put(ndrops - 1, 1, (double)nz);  // the drop reaches the wall z = nz
            close_drop(ndrops - 1, vol);
        }
    }
    out[0] = (double)ndrops;
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

cudaError_t launch_axis_drops(const double* fields, int nz, int nr, int zper, int max_drops, double* rows, double* out,
                              cudaStream_t st) {
    axis_drops_kernel<<<1, kAxisThreads, 0, st>>>(fields, nz, nr, zper, max_drops, rows, out);
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

// ---------------------------------------------------------------- FP64 pipe rate
// Throughput probe of the FP64 pipe (no paper counterpart): every thread runs
// kChains independent chains of dependent FP64 fused multiply-adds, enough
// independent work per warp to keep the pipe busy, and writes one sum so the
// work is not removed.  The rate is the FMA count over the CUDA-event time of
// the launch.
namespace {
constexpr int kFmaChains = 8;
__global__ void __launch_bounds__(256) dfma_rate_kernel(int iters, double a, double b, double* out) {
    double x[kFmaChains];
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c) x[c] = (double)(threadIdx.x + c) * 1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kFmaChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
}  // namespace

extern "C" int lbm_measure_fp64_rate(int32_t iters, void* stream, double* fma_per_second) {
    if (iters < 1 || !fma_per_second) return LBM_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    const int blocks = 4 * sms, threads = 256;
    double* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = LBM_OK;
    if (cudaMalloc(&out, (size_t)blocks * threads * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ERR_OOM;
    }
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = LBM_ERR_CUDA;
    // one warm-up launch, then the timed one
    for (int rep = 0; rep < 2 && rc == LBM_OK; ++rep) {
        if (rep == 1 && cudaEventRecord(e0, st) != cudaSuccess) rc = LBM_ERR_CUDA;
        dfma_rate_kernel<<<blocks, threads, 0, st>>>(iters, 0.999999, 1e-7, out);
        if (cudaGetLastError() != cudaSuccess) rc = LBM_ERR_CUDA;
        if (rep == 1 && rc == LBM_OK && cudaEventRecord(e1, st) != cudaSuccess) rc = LBM_ERR_CUDA;
    }
    float ms = 0.0f;
    if (rc == LBM_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        rc = LBM_ERR_CUDA;
    if (rc == LBM_OK) *fma_per_second = (double)blocks * threads * kFmaChains * (double)iters / (ms * 1e-3);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (rc != LBM_OK) cudaGetLastError();
    return rc;
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
