// lbm_capi.cu -- the C ABI of include/lbm.h: handle life cycle, device memory,
// step scheduling (direct launches and captured CUDA graphs), field and
// diagnostics read-back, state transfer, checkpoints and the launch-shape
// autotuner.  All numerical work is done by the kernels in lbm_kernels.cuh and
// lbm_diag.cu; this file only validates, allocates, launches and copies.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_device.cuh"
#include "lbm_internal.h"

using namespace axilbm;

namespace {

constexpr int kGraphSteps = 32;  // steps per captured graph (even: parity returns)
constexpr int kMax16BitNr = 65536;  // largest nr of the 16-bit storage forms

size_t pt_size(int prec) { return prec == LBM_FP64 ? 8 : (prec == LBM_FP32 ? 4 : 2); }
// f_0: FP64, the double-float ledger (FP32, bfloat16), or FP16's one exact FP32 ledger word
size_t f0_size(int prec) { return prec == LBM_MIX_FP16 ? 4 : 8; }
size_t real_size(int prec) { return prec == LBM_FP64 ? 8 : 4; }
// bytes of one storage block (32 nodes) in this precision
size_t block_bytes(int prec) {
    return (size_t)block_bytes_of((int)f0_size(prec), (int)pt_size(prec), (int)real_size(prec));
}

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

int validate(const lbm_params& p) {
    if (p.nr < 2 || p.nz < 2) return LBM_ERR_INVALID_ARG;
    // 32-bit node indices inside a case (nz * pitch), and 32-bit byte offsets
    // across one row of storage blocks
    if ((int64_t)p.nz * ((p.nr + 31) / 32 * 32) >= ((int64_t)1 << 31)) return LBM_ERR_INVALID_ARG;
    if ((int64_t)((p.nr + 31) / 32) * (int64_t)block_bytes(p.precision) >= ((int64_t)1 << 31))
        return LBM_ERR_INVALID_ARG;
    if (p.z_periodic != 0 && p.z_periodic != 1) return LBM_ERR_INVALID_ARG;
    if (p.precision < LBM_FP64 || p.precision > LBM_MIX_BF16) return LBM_ERR_INVALID_ARG;
    // 16-bit storage: the column scales P / 8 (P <= 2 nr) are FP16 numbers
    if ((p.precision == LBM_MIX_FP16 || p.precision == LBM_MIX_BF16) && p.nr > kMax16BitNr)
        return LBM_ERR_INVALID_ARG;
    if (p.p_coupling != LBM_P_EXACT && p.p_coupling != LBM_P_LAGGED) return LBM_ERR_INVALID_ARG;
    if (p.collision != LBM_MRT_ORTHOGONAL && p.collision != LBM_MRT_RAW) return LBM_ERR_INVALID_ARG;
    if (!finite_pos(p.rho_l) || !finite_pos(p.rho_g) || !finite_pos(p.nu_l) || !finite_pos(p.nu_g))
        return LBM_ERR_INVALID_ARG;
    if (!finite_pos(p.W) || !finite_pos(p.mobility)) return LBM_ERR_INVALID_ARG;
    if (!std::isfinite(p.sigma) || p.sigma < 0.0 || !std::isfinite(p.grav_z)) return LBM_ERR_INVALID_ARG;
    if (!std::isfinite(p.n_eps) || p.n_eps < 0.0) return LBM_ERR_INVALID_ARG;
    for (int i = 0; i < 9; ++i) {
        for (double s : {p.sf[i], p.sg[i]}) {
            if (!std::isfinite(s)) return LBM_ERR_INVALID_ARG;
            if (s >= 0.0 && s >= 2.0) return LBM_ERR_INVALID_ARG;
        }
    }
    return LBM_OK;
}

int nargs_of(int shape) {
    switch (shape) {
        case LBM_SHAPE_FLAT: return 3;
        case LBM_SHAPE_SPHERE: return 3;
        case LBM_SHAPE_ELLIPSOID: return 4;
        case LBM_SHAPE_P2: return 4;
        case LBM_SHAPE_THREAD: return 5;
        case LBM_SHAPE_BUBBLE: return 3;
        case LBM_SHAPE_HOST_ARRAY: return 0;
        default: return -1;
    }
}

}  // namespace

struct lbm_sim {
    int device = 0;
    int precision = 0;
    int ncases = 0;
    cudaStream_t stream = nullptr;      // caller's stream
    cudaStream_t cap_stream = nullptr;  // private stream used for graph capture
    std::vector<lbm_params> prm;
    std::vector<CaseDev> cases;
    std::vector<int64_t> case_steps;
    std::vector<char> initialized;
    DeviceState D{};
    // tiles: one list per step variant over all cases, plus the 8-row tiling
    // of each case for the field kernel
    TileDev* tiles_d[kNumVariants] = {};
    int ntiles[kNumVariants] = {};
    std::vector<TileDev*> ftiles_d;
    std::vector<int> nftiles;
    int64_t max_nodes = 0;  // largest nz * nr of a case
    double* fields = nullptr;   // [5][nz][nr] of the largest case
    double* phi0 = nullptr;     // [nz][nr]
    double* phi0_all = nullptr;  // every case's [nz][nr], made by the first lbm_init_phase_all
    double* state = nullptr;    // [21][nz][nr]
    double* partials = nullptr;
    double* diag_out = nullptr;
    double* axis_rows = nullptr;   // nz doubles of the tallest case
    double* axis_out = nullptr;    // the drops record, 3 + 4 * kMaxAxisDrops doubles
    double* axis_host = nullptr;   // pinned copy of axis_out
    // pinned host staging for small reads (a diagnostics record and the
    // status word), so that they return with one synchronisation
    double* host_small = nullptr;
    // pipelined diagnostics: per slot a completion event, the caller's record
    // and a pinned copy of the device status word
    cudaEvent_t diag_ev[LBM_DIAG_SLOTS] = {};
    lbm_diag* slot_out[LBM_DIAG_SLOTS] = {};
    int* slot_status = nullptr;
    // Pipelined diagnostics run on a private stream beside the next steps:
    // ev_state marks the state they read, ev_fields the end of that read (the
    // handle's stream waits for it before it overwrites the state), ev_diag
    // the end of their use of the shared scratch (fields, partials, record),
    // which the handle's stream joins before it uses that scratch itself.
    cudaStream_t diag_stream = nullptr;
    cudaEvent_t ev_state = nullptr, ev_fields = nullptr, ev_diag = nullptr;
    bool diag_pending = false;
    std::vector<void*> allocations;
    int parity = 0;
    int variant = 0;
    int sticky = LBM_OK;
    int64_t launches = 0;
    cudaGraphExec_t graph = nullptr;
    int graph_variant = -1;
    bool tma_ok = false;  // tensor maps could be encoded for every case
};

namespace {

int fail(lbm_sim* h, int code) {
    if (code == LBM_ERR_CUDA || code == LBM_ERR_NONFINITE) h->sticky = code;
    return code;
}

int cuda_ok(lbm_sim* h, cudaError_t e) {
    if (e == cudaSuccess) return LBM_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return LBM_ERR_OOM;
    }
    return fail(h, LBM_ERR_CUDA);
}

cudaError_t dev_alloc(lbm_sim* h, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 256;
    cudaError_t e = cudaMallocAsync(p, bytes, h->stream);
    if (e != cudaSuccess) return e;
    h->allocations.push_back(*p);
    return cudaMemsetAsync(*p, 0, bytes, h->stream);
}

cudaError_t launch_step_any(lbm_sim* h, int parity, int variant, cudaStream_t st) {
    const TileDev* t = h->tiles_d[variant];
    const int n = h->ntiles[variant];
    switch (h->precision) {
        case LBM_FP64: return launch_step_f64(h->D, parity, variant, t, n, st);
        case LBM_FP32: return launch_step_f32(h->D, parity, variant, t, n, st);
        case LBM_MIX_FP16: return launch_step_h16(h->D, parity, variant, t, n, st);
        default: return launch_step_b16(h->D, parity, variant, t, n, st);
    }
}

cudaError_t launch_fields_any(lbm_sim* h, int icase, cudaStream_t st) {
    const TileDev* t = h->ftiles_d[icase];
    const int n = h->nftiles[icase];
    switch (h->precision) {
        case LBM_FP64: return launch_fields_f64(h->D, h->parity, t, n, h->fields, st);
        case LBM_FP32: return launch_fields_f32(h->D, h->parity, t, n, h->fields, st);
        case LBM_MIX_FP16: return launch_fields_h16(h->D, h->parity, t, n, h->fields, st);
        default: return launch_fields_b16(h->D, h->parity, t, n, h->fields, st);
    }
}

// Initial condition from dense phi0: of case icase alone (phi0 holds its
// [nz][nr]), or with icase < 0 of every case (phi0 holds all of them in order).
cudaError_t launch_init_any(lbm_sim* h, int icase, const double* phi0) {
    const TileDev* t = icase < 0 ? h->tiles_d[0] : h->ftiles_d[icase];
    const int n = icase < 0 ? h->ntiles[0] : h->nftiles[icase];
    const int64_t base = icase < 0 ? 0 : h->cases[icase].dense_off;
    static_assert(kVariantTZ[0] == 8, "the initial condition covers 8-row tiles");
    switch (h->precision) {
        case LBM_FP64: return launch_init_f64(h->D, h->parity, t, n, phi0, base, h->stream);
        case LBM_FP32: return launch_init_f32(h->D, h->parity, t, n, phi0, base, h->stream);
        case LBM_MIX_FP16: return launch_init_h16(h->D, h->parity, t, n, phi0, base, h->stream);
        default: return launch_init_b16(h->D, h->parity, t, n, phi0, base, h->stream);
    }
}

cudaError_t launch_get_state_any(lbm_sim* h, int icase, double* f, double* g, double* aux) {
    const CaseDev& C = h->cases[icase];
    switch (h->precision) {
        case LBM_FP64: return launch_get_state_f64(h->D, h->parity, C, f, g, aux, h->stream);
        case LBM_FP32: return launch_get_state_f32(h->D, h->parity, C, f, g, aux, h->stream);
        case LBM_MIX_FP16: return launch_get_state_h16(h->D, h->parity, C, f, g, aux, h->stream);
        default: return launch_get_state_b16(h->D, h->parity, C, f, g, aux, h->stream);
    }
}

cudaError_t launch_set_state_any(lbm_sim* h, int icase, const double* f, const double* g, const double* aux) {
    const CaseDev& C = h->cases[icase];
    switch (h->precision) {
        case LBM_FP64: return launch_set_state_f64(h->D, h->parity, C, f, g, aux, h->stream);
        case LBM_FP32: return launch_set_state_f32(h->D, h->parity, C, f, g, aux, h->stream);
        case LBM_MIX_FP16: return launch_set_state_h16(h->D, h->parity, C, f, g, aux, h->stream);
        default: return launch_set_state_b16(h->D, h->parity, C, f, g, aux, h->stream);
    }
}

template <typename Real>
void fill_params(CaseReal<Real>& P, const lbm_params& p) {
    P.rho_l = (Real)p.rho_l;
    P.rho_g = (Real)p.rho_g;
    P.nu_l = (Real)p.nu_l;
    P.nu_g = (Real)p.nu_g;
    P.grav_z = (Real)p.grav_z;
    P.n_eps = (Real)p.n_eps;
    P.beta = (Real)(12.0 * p.sigma / p.W);  // Eq. 4
    P.kappa = (Real)(1.5 * p.sigma * p.W);
    P.inv_W = (Real)(1.0 / p.W);
    P.mob = (Real)p.mobility;
    const double inv_tau_f = 1.0 / (p.mobility * 3.0 + 0.5);  // Eq. 18
    for (int i = 0; i < 9; ++i) {
        P.sf[i] = (Real)(p.sf[i] < 0.0 ? inv_tau_f : p.sf[i]);
        P.sg[i] = (Real)(p.sg[i] < 0.0 ? 0.0 : p.sg[i]);
    }
}

// The rate pattern of a case, when the kernels know it at compile time
// (kRatesPaper / kRatesPaperRaw in lbm_internal.h), else kRatesGeneral.
// Orthogonal moments, the paper's runs (Sec. 3.1): S^f = diag(1, 1, 1, s, s,
// s, s, 1, 1) with one s; S^g = 1 except s1 = s7 = s8 derived from the local
// viscosity.  Raw moments: S^f = 1 except one s on moments 1, 2, 6, 7; S^g = 1
// except 3, 4, 5 derived from the local viscosity.
int rate_pattern(const lbm_params& p) {
    const bool raw = p.collision == LBM_MRT_RAW;
    const int fs = raw ? 1 : 3;  // index of the f moment that carries s
    for (int i = 0; i < 9; ++i) {
        const bool s_f = raw ? (i == 1 || i == 2 || i == 6 || i == 7) : (i >= 3 && i <= 6);
        if (s_f ? (p.sf[i] != p.sf[fs]) : (p.sf[i] != 1.0)) return kRatesGeneral;
        const bool local = raw ? (i >= 3 && i <= 5) : (i == 1 || i == 7 || i == 8);
        if (local ? !(p.sg[i] < 0.0) : (p.sg[i] != 1.0)) return kRatesGeneral;
    }
    return raw ? kRatesPaperRaw : kRatesPaper;
}

CaseDev make_case(const lbm_params& p, int64_t off, int64_t dense_off) {
    CaseDev C{};
    C.dense_off = dense_off;
    C.nr = p.nr;
    C.nz = p.nz;
    C.pitch = (p.nr + 31) / 32 * 32;
    C.plane = p.nz * C.pitch;
    C.zper = p.z_periodic;
    C.p_coupling = p.p_coupling;
    C.collision = p.collision;
    C.off = off;
    C.sg_local = 0;
    for (int i = 0; i < 9; ++i)
        if (p.sg[i] < 0.0) C.sg_local |= 1u << i;
    fill_params<double>(C.pd, p);
    fill_params<float>(C.pf, p);
    return C;
}

std::vector<TileDev> make_tiles(const std::vector<CaseDev>& cs, int tz, int only_case) {
    std::vector<TileDev> t;
    for (int c = 0; c < (int)cs.size(); ++c) {
        if (only_case >= 0 && c != only_case) continue;
        for (int k0 = 0; k0 < cs[c].nz; k0 += tz)
            for (int j0 = 0; j0 < cs[c].nr; j0 += 32) t.push_back(TileDev{c, k0, j0, 0});
    }
    return t;
}

// A tile list on the device; with geo, followed by one TileGeo per tile (the
// step variants' lists).
int upload_tiles(lbm_sim* h, const std::vector<TileDev>& t, TileDev** out, bool geo = false) {
    static_assert(sizeof(TileDev) == 16 && sizeof(TileGeo) == 32, "tile record sizes");
    std::vector<TileGeo> g;
    if (geo) {
        g.reserve(t.size());
        for (const TileDev& d : t) {
            const CaseDev& C = h->cases[d.c];
            g.push_back(TileGeo{d.c, d.k0, d.j0, (int32_t)(C.off >> 5), C.pitch >> 5, C.nr, C.nz, C.zper});
        }
    }
    void* p = nullptr;
    const size_t tb = t.size() * sizeof(TileDev), gb = g.size() * sizeof(TileGeo);
    cudaError_t e = dev_alloc(h, &p, std::max<size_t>(1, tb + gb));
    if (e != cudaSuccess) return cuda_ok(h, e);
    if (!t.empty()) {
        e = cudaMemcpyAsync(p, t.data(), tb, cudaMemcpyHostToDevice, h->stream);
        if (e != cudaSuccess) return cuda_ok(h, e);
    }
    if (!g.empty()) {
        e = cudaMemcpyAsync((char*)p + tb, g.data(), gb, cudaMemcpyHostToDevice, h->stream);
        if (e != cudaSuccess) return cuda_ok(h, e);
        // the host vectors are pageable: each copy has been staged when it returns
    }
    *out = (TileDev*)p;
    return LBM_OK;
}

void release(lbm_sim* h) {
    if (h->graph) cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
    for (void* p : h->allocations) cudaFreeAsync(p, h->stream);
    h->allocations.clear();
    // every copy still pending into the pinned buffers below ends here
    cudaStreamSynchronize(h->stream);
    if (h->diag_stream) cudaStreamSynchronize(h->diag_stream);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    h->cap_stream = nullptr;
    if (h->diag_stream) cudaStreamDestroy(h->diag_stream);
    h->diag_stream = nullptr;
    for (cudaEvent_t* e : {&h->ev_state, &h->ev_fields, &h->ev_diag}) {
        if (*e) cudaEventDestroy(*e);
        *e = nullptr;
    }
    if (h->host_small) cudaFreeHost(h->host_small);
    h->host_small = nullptr;
    if (h->slot_status) cudaFreeHost(h->slot_status);
    h->slot_status = nullptr;
    if (h->axis_host) cudaFreeHost(h->axis_host);
    h->axis_host = nullptr;
    for (cudaEvent_t& e : h->diag_ev) {
        if (e) cudaEventDestroy(e);
        e = nullptr;
    }
}

// Tensor maps of the step's storage blocks (kMapsPerCase per case and per tile
// height of 8 and 16 rows): the TMA-pipelined step stages boxes of the tile's
// rows plus two above and below, and the register-path step prefetches boxes
// of the tile's own rows into L2.  Returns false when the driver entry point
// is missing or a map is rejected; the TMA variants and the prefetch are then
// unused.
bool encode_tensor_maps(lbm_sim* h, std::vector<CUtensorMap>& maps) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn) {
            cudaGetLastError();
            return false;
        }
        encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    const int p = h->precision;
    const size_t B = block_bytes(p);
    maps.assign((size_t)h->ncases * 2 * kMapsPerCase, CUtensorMap{});
    for (int c = 0; c < h->ncases; ++c) {
        const CaseDev& C = h->cases[c];
        const int ng = C.pitch / 32;
        for (int set = 0; set < 2; ++set) {
            const cuuint32_t tz = set == 0 ? 8 : 16;
            CUtensorMap* M = &maps[((size_t)c * 2 + set) * kMapsPerCase];
            // the case's blocks as 32-bit words: [rows][column groups][128-byte slots][32 words];
            // a box is tz + 4 rows (staging) or tz rows (prefetch) of one column group, every slot
            for (int m = 0; m < 4; ++m) {
                const int b = m & 1;
                void* base = (char*)h->D.blk[b] + (size_t)(C.off / 32) * B;
                const cuuint64_t dims[4] = {32, (cuuint64_t)(B / 128), (cuuint64_t)ng, (cuuint64_t)C.nz};
                const cuuint64_t strides[3] = {128, (cuuint64_t)B, (cuuint64_t)ng * B};
                const cuuint32_t box[4] = {32, (cuuint32_t)(B / 128), 1, m < 2 ? tz + 4 : tz};
                const cuuint32_t estr[4] = {1, 1, 1, 1};
                if (encode(M + m, CU_TENSOR_MAP_DATA_TYPE_UINT32, 4, base, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                    return false;
            }
        }
    }
    return true;
}

int create_impl(const lbm_params* cases, int32_t n, void* stream, lbm_handle** out) {
    if (!out) return LBM_ERR_INVALID_ARG;
    *out = nullptr;
    if (!cases || n < 1) return LBM_ERR_INVALID_ARG;
    for (int c = 0; c < n; ++c) {
        int v = validate(cases[c]);
        if (v != LBM_OK) return v;
        if (cases[c].precision != cases[0].precision) return LBM_ERR_INVALID_ARG;
    }
    lbm_sim* h = new (std::nothrow) lbm_sim();
    if (!h) return LBM_ERR_OOM;
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return LBM_ERR_CUDA;
    }
    h->stream = (cudaStream_t)stream;
    h->precision = cases[0].precision;
    h->ncases = n;
    h->prm.assign(cases, cases + n);
    int64_t off = 0, dense = 0;
    int max_nz = 0;
    for (int c = 0; c < n; ++c) {
        max_nz = std::max(max_nz, cases[c].nz);
        h->cases.push_back(make_case(cases[c], off, dense));
        dense += (int64_t)cases[c].nz * cases[c].nr;
        off += (int64_t)h->cases[c].nz * h->cases[c].pitch;
        h->max_nodes = std::max<int64_t>(h->max_nodes, (int64_t)cases[c].nz * cases[c].nr);
    }
    h->D.total = off;
    // one rate mode for the whole handle: the pattern all cases share, else general
    h->D.rate_mode = rate_pattern(cases[0]);
    for (int c = 1; c < n; ++c)
        if (rate_pattern(cases[c]) != h->D.rate_mode) h->D.rate_mode = kRatesGeneral;
    h->case_steps.assign(n, 0);
    h->initialized.assign(n, 0);
    int rc = LBM_OK;
    auto A = [&](void** p, size_t bytes) {
        if (rc != LBM_OK) return;
        cudaError_t e = dev_alloc(h, p, bytes);
        if (e != cudaSuccess) rc = (e == cudaErrorMemoryAllocation) ? LBM_ERR_OOM : LBM_ERR_CUDA;
    };
    const size_t T = (size_t)off;
    for (int b = 0; b < 2; ++b) {
        A(&h->D.blk[b], (T / 32) * block_bytes(h->precision));
    }
    A(&h->D.cases, n * sizeof(CaseDev));
    A((void**)&h->fields, 5 * (size_t)h->max_nodes * sizeof(double));
    A((void**)&h->phi0, (size_t)h->max_nodes * sizeof(double));
    A((void**)&h->state, 21 * (size_t)h->max_nodes * sizeof(double));
    A((void**)&h->partials, diag_partials_size() * sizeof(double));
    A((void**)&h->diag_out, 16 * sizeof(double));
    A((void**)&h->axis_rows, (size_t)max_nz * sizeof(double));
    A((void**)&h->axis_out, (3 + 4 * kMaxAxisDrops) * sizeof(double));
    A((void**)&h->D.status, 128);
    if (rc == LBM_OK && cudaMallocHost((void**)&h->host_small, 16 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        h->host_small = nullptr;
        rc = LBM_ERR_OOM;
    }
    if (rc == LBM_OK && cudaMallocHost((void**)&h->axis_host, (3 + 4 * kMaxAxisDrops) * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        h->axis_host = nullptr;
        rc = LBM_ERR_OOM;
    }
    if (rc == LBM_OK && cudaMallocHost((void**)&h->slot_status, LBM_DIAG_SLOTS * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        h->slot_status = nullptr;
        rc = LBM_ERR_OOM;
    }
    for (int q = 0; q < LBM_DIAG_SLOTS && rc == LBM_OK; ++q)
        if (cudaEventCreateWithFlags(&h->diag_ev[q], cudaEventDisableTiming) != cudaSuccess) rc = LBM_ERR_CUDA;
    for (cudaEvent_t* e : {&h->ev_state, &h->ev_fields, &h->ev_diag})
        if (rc == LBM_OK && cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) rc = LBM_ERR_CUDA;
    // the diagnostics stream has the greatest priority, so that its few blocks
    // are scheduled ahead of the next step's tiles instead of after them
    if (rc == LBM_OK) {
        int least = 0, greatest = 0;
        if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess ||
            cudaStreamCreateWithPriority(&h->diag_stream, cudaStreamNonBlocking, greatest) != cudaSuccess)
            rc = LBM_ERR_CUDA;
    }
    if (rc == LBM_OK) {
        std::vector<CUtensorMap> maps;
        h->tma_ok = encode_tensor_maps(h, maps);
        if (h->tma_ok) {
            void* dm = nullptr;
            A(&dm, maps.size() * sizeof(CUtensorMap));
            if (rc == LBM_OK && cudaMemcpyAsync(dm, maps.data(), maps.size() * sizeof(CUtensorMap),
                                                cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
                rc = LBM_ERR_CUDA;
            h->D.tmaps = dm;
        }
    }
    if (rc == LBM_OK) {
        cudaError_t e = cudaMemcpyAsync(h->D.cases, h->cases.data(), n * sizeof(CaseDev), cudaMemcpyHostToDevice,
                                        h->stream);
        if (e != cudaSuccess) rc = LBM_ERR_CUDA;
    }
    for (int v = 0; v < kNumVariants && rc == LBM_OK; ++v) {
        std::vector<TileDev> t = make_tiles(h->cases, kVariantTZ[v], -1);
        h->ntiles[v] = (int)t.size();
        rc = upload_tiles(h, t, &h->tiles_d[v], true);
    }
    for (int c = 0; c < n && rc == LBM_OK; ++c) {
        std::vector<TileDev> t = make_tiles(h->cases, 8, c);
        TileDev* d = nullptr;
        rc = upload_tiles(h, t, &d);
        h->ftiles_d.push_back(d);
        h->nftiles.push_back((int)t.size());
    }
    if (rc == LBM_OK && cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        rc = LBM_ERR_CUDA;
    if (rc == LBM_OK && cudaStreamSynchronize(h->stream) != cudaSuccess) rc = LBM_ERR_CUDA;
    if (rc != LBM_OK) {
        cudaGetLastError();
        release(h);
        delete h;
        return rc;
    }
    *out = h;
    return LBM_OK;
}

int enter(lbm_sim* h) {
    if (!h) return LBM_ERR_INVALID_ARG;
    if (h->sticky != LBM_OK) return h->sticky;
    if (cudaSetDevice(h->device) != cudaSuccess) return fail(h, LBM_ERR_CUDA);
    return LBM_OK;
}

int capture_graph(lbm_sim* h) {
    if (h->graph && h->graph_variant == h->variant) return LBM_OK;
    if (h->graph) cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return fail(h, LBM_ERR_CUDA);
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < kGraphSteps && e == cudaSuccess; ++s) e = launch_step_any(h, s & 1, h->variant, h->cap_stream);
    cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return fail(h, LBM_ERR_CUDA);
    }
    e = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        h->graph = nullptr;
        return fail(h, LBM_ERR_CUDA);
    }
    h->graph_variant = h->variant;
    return LBM_OK;
}

int step_direct(lbm_sim* h, int64_t n) {
    for (int64_t s = 0; s < n; ++s) {
        cudaError_t e = launch_step_any(h, h->parity, h->variant, h->stream);
        if (e != cudaSuccess) return cuda_ok(h, e);
        h->parity ^= 1;
        h->launches += 1;
    }
    return LBM_OK;
}

// Device status word: set by a bounded wait that gave up (TMA-staged step).
int check_status(lbm_sim* h) {
    int st = 0;
    if (cudaMemcpyAsync(&st, h->D.status, sizeof(int), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
        return fail(h, LBM_ERR_CUDA);
    if (st != 0) {
        h->sticky = LBM_ERR_TIMEOUT;
        return LBM_ERR_TIMEOUT;
    }
    return LBM_OK;
}

int check_case(lbm_sim* h, int icase) {
    if (icase < 0 || icase >= h->ncases) return LBM_ERR_INVALID_ARG;
    return LBM_OK;
}

// Order the handle's stream after the pipelined diagnostics' use of the
// shared scratch (fields, partials, record) before it uses that scratch.
int join_diagnostics(lbm_sim* h) {
    if (!h->diag_pending) return LBM_OK;
    int rc = cuda_ok(h, cudaStreamWaitEvent(h->stream, h->ev_diag, 0));
    if (rc == LBM_OK) h->diag_pending = false;
    return rc;
}

// Enqueue the fields and the reductions of case icase, then the copies of the
// 11-double record to `record` and of the device status word to `status`
// (host memory), on stream `st`.  When st is the diagnostics stream, the
// fields' read of the state is ordered after the work already on the handle's
// stream, and the handle's stream waits for that read only.  Does not wait.
int enqueue_diagnostics(lbm_sim* h, int icase, double* record, int* status, cudaStream_t st) {
    const bool side = st != h->stream;
    int rc = LBM_OK;
    if (side) {
        rc = cuda_ok(h, cudaEventRecord(h->ev_state, h->stream));
        if (rc == LBM_OK) rc = cuda_ok(h, cudaStreamWaitEvent(st, h->ev_state, 0));
    } else {
        rc = join_diagnostics(h);
    }
    if (rc != LBM_OK) return rc;
    rc = cuda_ok(h, launch_fields_any(h, icase, st));
    if (rc != LBM_OK) return rc;
    if (side) {
        rc = cuda_ok(h, cudaEventRecord(h->ev_fields, st));
        if (rc == LBM_OK) rc = cuda_ok(h, cudaStreamWaitEvent(h->stream, h->ev_fields, 0));
        if (rc != LBM_OK) return rc;
    }
    const lbm_params& p = h->prm[icase];
    rc = cuda_ok(h, launch_diag(h->fields, p.nz, p.nr, p.z_periodic, (double)h->case_steps[icase], h->partials,
                                h->diag_out, st));
    if (rc != LBM_OK) return rc;
    rc = cuda_ok(h, cudaMemcpyAsync(record, h->diag_out, 11 * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (rc != LBM_OK) return rc;
    rc = cuda_ok(h, cudaMemcpyAsync(status, h->D.status, sizeof(int), cudaMemcpyDeviceToHost, st));
    if (rc != LBM_OK || !side) return rc;
    rc = cuda_ok(h, cudaEventRecord(h->ev_diag, st));
    if (rc == LBM_OK) h->diag_pending = true;
    return rc;
}

}  // namespace

extern "C" {

int lbm_create(const lbm_params* prm, void* stream, lbm_handle** out) { return create_impl(prm, 1, stream, out); }

int lbm_batch_create(const lbm_params* cases, int32_t ncases, void* stream, lbm_handle** out) {
    return create_impl(cases, ncases, stream, out);
}

int32_t lbm_num_cases(const lbm_handle* h) { return h ? h->ncases : 0; }

int lbm_case_init_phase(lbm_handle* h, int32_t icase, int32_t shape, const double* shape_args, int32_t nargs,
                        const double* host_phi) {
    int rc = enter(h);
    if (rc != LBM_OK) return rc;
    if (check_case(h, icase) != LBM_OK) return LBM_ERR_INVALID_ARG;
    const int need = nargs_of(shape);
    if (need < 0) return LBM_ERR_INVALID_ARG;
    const lbm_params& p = h->prm[icase];
    const int64_t n = (int64_t)p.nz * p.nr;
    if (shape == LBM_SHAPE_HOST_ARRAY) {
        if (!host_phi) return LBM_ERR_INVALID_ARG;
        rc = cuda_ok(h, cudaMemcpyAsync(h->phi0, host_phi, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    } else {
        if (nargs != need || !shape_args) return LBM_ERR_INVALID_ARG;
        for (int i = 0; i < nargs; ++i)
            if (!std::isfinite(shape_args[i])) return LBM_ERR_INVALID_ARG;
        rc = cuda_ok(h, launch_shape(shape, shape_args, nargs, p.nz, p.nr, h->phi0, h->stream));
    }
    if (rc != LBM_OK) return rc;
    rc = cuda_ok(h, launch_init_any(h, icase, h->phi0));
    if (rc != LBM_OK) return rc;
    h->case_steps[icase] = 0;
    h->initialized[icase] = 1;
    return cuda_ok(h, cudaStreamSynchronize(h->stream));
}

int lbm_init_phase_all(lbm_handle* h, const double* host_phi) {
    int rc = enter(h);
    if (rc != LBM_OK) return rc;
    if (!host_phi) return LBM_ERR_INVALID_ARG;
    int64_t total = 0;
    for (const lbm_params& p : h->prm) total += (int64_t)p.nz * p.nr;
    if (!h->phi0_all) {
        void* p = nullptr;
        rc = cuda_ok(h, dev_alloc(h, &p, (size_t)total * sizeof(double)));
        if (rc != LBM_OK) return rc;
        h->phi0_all = (double*)p;
    }
    rc = cuda_ok(h, cudaMemcpyAsync(h->phi0_all, host_phi, (size_t)total * sizeof(double), cudaMemcpyHostToDevice,
                                    h->stream));
    // one launch over the 8-row tiles of every case
    if (rc == LBM_OK) rc = cuda_ok(h, launch_init_any(h, -1, h->phi0_all));
    if (rc != LBM_OK) return rc;
    for (int c = 0; c < h->ncases; ++c) {
        h->case_steps[c] = 0;
        h->initialized[c] = 1;
    }
    return cuda_ok(h, cudaStreamSynchronize(h->stream));
}

int lbm_init_phase(lbm_handle* h, int32_t shape, const double* shape_args, int32_t nargs, const double* host_phi) {
    return lbm_case_init_phase(h, 0, shape, shape_args, nargs, host_phi);
}

int lbm_step(lbm_handle* h, int64_t nsteps) {
    int rc = enter(h);
    if (rc != LBM_OK) return rc;
    if (nsteps < 0) return LBM_ERR_INVALID_ARG;
    for (int c = 0; c < h->ncases; ++c)
        if (!h->initialized[c]) return LBM_ERR_STATE;
    if (nsteps == 0) return LBM_OK;
    int64_t left = nsteps;
    if (left >= kGraphSteps) {
        if (h->parity == 1) {
            rc = step_direct(h, 1);
            if (rc != LBM_OK) return rc;
            left -= 1;
        }
        if (left >= kGraphSteps) {
            rc = capture_graph(h);
            if (rc != LBM_OK) return rc;
            while (left >= kGraphSteps) {
                cudaError_t e = cudaGraphLaunch(h->graph, h->stream);
                if (e != cudaSuccess) return cuda_ok(h, e);
                left -= kGraphSteps;
                h->launches += kGraphSteps;
            }
        }
    }
    rc = step_direct(h, left);
    if (rc != LBM_OK) return rc;
    for (int c = 0; c < h->ncases; ++c) h->case_steps[c] += nsteps;
    return LBM_OK;
}

int lbm_case_get_fields(lbm_handle* h, int32_t icase, int32_t mask, double* host_out) {
    int rc = enter(h);
    if (rc != LBM_OK) return rc;
    if (check_case(h, icase) != LBM_OK || !host_out || mask <= 0 || mask > 31) return LBM_ERR_INVALID_ARG;
    if (!h->initialized[icase]) return LBM_ERR_STATE;
    rc = check_status(h);
    if (rc != LBM_OK) return rc;
    rc = join_diagnostics(h);
    if (rc != LBM_OK) return rc;
    rc = cuda_ok(h, launch_fields_any(h, icase, h->stream));
    if (rc != LBM_OK) return rc;
    const int64_t n = (int64_t)h->prm[icase].nz * h->prm[icase].nr;
    int slot = 0;
    for (int b = 0; b < 5; ++b) {
        if (!(mask & (1 << b))) continue;
        rc = cuda_ok(h, cudaMemcpyAsync(host_out + slot * n, h->fields + b * n, n * sizeof(double),
                                        cudaMemcpyDeviceToHost, h->stream));
        if (rc != LBM_OK) return rc;
        ++slot;
    }
    return cuda_ok(h, cudaStreamSynchronize(h->stream));
}

int lbm_get_fields(lbm_handle* h, int32_t mask, double* host_out) { return lbm_case_get_fields(h, 0, mask, host_out); }

int lbm_case_diagnostics(lbm_handle* h, int32_t icase, lbm_diag* out) {
    int rc = enter(h);
    if (rc != LBM_OK) return rc;
    if (check_case(h, icase) != LBM_OK || !out) return LBM_ERR_INVALID_ARG;
    if (!h->initialized[icase]) return LBM_ERR_STATE;
    // the record and the device status word come back with one synchronisation
    double* buf = h->host_small;          // 11 doubles of the record
    int* st_h = (int*)(h->host_small + 12);  // the status word
    rc = enqueue_diagnostics(h, icase, buf, st_h, h->stream);
    if (rc != LBM_OK) return rc;
    rc = cuda_ok(h, cudaStreamSynchronize(h->stream));
    if (rc != LBM_OK) return rc;
    if (*st_h != 0) {
        h->sticky = LBM_ERR_TIMEOUT;
        return LBM_ERR_TIMEOUT;
    }
    static_assert(sizeof(lbm_diag) == 11 * sizeof(double), "diag layout");
    std::memcpy(out, buf, sizeof(lbm_diag));
    if (out->nonfinite > 0) return fail(h, LBM_ERR_NONFINITE);
    return LBM_OK;
}

int lbm_diagnostics(lbm_handle* h, lbm_diag* out) { return lbm_case_diagnostics(h, 0, out); }

int lbm_case_axis_drops(lbm_handle* h, int32_t icase, int32_t max_drops, lbm_drop* drops, int32_t* n_drops,
                        double* axis_min) {
    static_assert(sizeof(lbm_drop) == 4 * sizeof(double), "drop record layout");
    static_assert(LBM_MAX_AXIS_DROPS == kMaxAxisDrops, "drop capacity");
    int rc = enter(h);
    if (rc != LBM_OK) return rc;
    if (check_case(h, icase) != LBM_OK || !n_drops || max_drops < 0 || max_drops > kMaxAxisDrops ||
        (max_drops > 0 && !drops))
        return LBM_ERR_INVALID_ARG;
    if (!h->initialized[icase]) return LBM_ERR_STATE;
    rc = check_status(h);
    if (rc != LBM_OK) return rc;
    rc = join_diagnostics(h);
    if (rc != LBM_OK) return rc;
    rc = cuda_ok(h, launch_fields_any(h, icase, h->stream));
    if (rc != LBM_OK) return rc;
    const lbm_params& p = h->prm[icase];
    rc = cuda_ok(h, launch_axis_drops(h->fields, p.nz, p.nr, p.z_periodic, max_drops, h->axis_rows, h->axis_out,
                                      h->stream));
    if (rc != LBM_OK) return rc;
    rc = cuda_ok(h, cudaMemcpyAsync(h->axis_host, h->axis_out, (3 + 4 * (size_t)max_drops) * sizeof(double),
                                    cudaMemcpyDeviceToHost, h->stream));
    if (rc != LBM_OK) return rc;
    rc = cuda_ok(h, cudaStreamSynchronize(h->stream));
    if (rc != LBM_OK) return rc;
    const int n = (int)h->axis_host[0];
    *n_drops = n;
    if (axis_min) {
        axis_min[0] = h->axis_host[1];
        axis_min[1] = h->axis_host[2];
    }
    const int m = n < max_drops ? n : max_drops;
    if (m > 0) std::memcpy(drops, h->axis_host + 3, (size_t)m * sizeof(lbm_drop));
    return LBM_OK;
}

int lbm_case_diagnostics_enqueue(lbm_handle* h, int32_t icase, lbm_diag* host_out, int32_t slot) {
    int rc = enter(h);
    if (rc != LBM_OK) return rc;
    if (check_case(h, icase) != LBM_OK || !host_out || slot < 0 || slot >= LBM_DIAG_SLOTS) return LBM_ERR_INVALID_ARG;
    if (!h->initialized[icase]) return LBM_ERR_STATE;
    rc = enqueue_diagnostics(h, icase, (double*)host_out, h->slot_status + slot, h->diag_stream);
    if (rc != LBM_OK) return rc;
    rc = cuda_ok(h, cudaEventRecord(h->diag_ev[slot], h->diag_stream));
    if (rc != LBM_OK) return rc;
    h->slot_out[slot] = host_out;
    return LBM_OK;
}

int lbm_diagnostics_wait(lbm_handle* h, int32_t slot) {
    int rc = enter(h);
    if (rc != LBM_OK) return rc;
    if (slot < 0 || slot >= LBM_DIAG_SLOTS) return LBM_ERR_INVALID_ARG;
    lbm_diag* out = h->slot_out[slot];
    if (!out) return LBM_ERR_STATE;
    rc = cuda_ok(h, cudaEventSynchronize(h->diag_ev[slot]));
    if (rc != LBM_OK) return rc;
    h->slot_out[slot] = nullptr;
    if (h->slot_status[slot] != 0) {
        h->sticky = LBM_ERR_TIMEOUT;
        return LBM_ERR_TIMEOUT;
    }
    if (out->nonfinite > 0) return fail(h, LBM_ERR_NONFINITE);
    return LBM_OK;
}

int lbm_get_state(lbm_handle* h, int32_t icase, double* f, double* g, double* aux) {
    int rc = enter(h);
    if (rc != LBM_OK) return rc;
    if (check_case(h, icase) != LBM_OK) return LBM_ERR_INVALID_ARG;
    const int64_t n = (int64_t)h->prm[icase].nz * h->prm[icase].nr;
    double* df = h->state;
    double* dg = h->state + 9 * n;
    double* da = h->state + 18 * n;
    rc = cuda_ok(h, launch_get_state_any(h, icase, f ? df : nullptr, g ? dg : nullptr, aux ? da : nullptr));
    if (rc != LBM_OK) return rc;
    if (f) rc = cuda_ok(h, cudaMemcpyAsync(f, df, 9 * n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (rc == LBM_OK && g)
        rc = cuda_ok(h, cudaMemcpyAsync(g, dg, 9 * n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (rc == LBM_OK && aux)
        rc = cuda_ok(h, cudaMemcpyAsync(aux, da, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (rc != LBM_OK) return rc;
    return cuda_ok(h, cudaStreamSynchronize(h->stream));
}

int lbm_set_state(lbm_handle* h, int32_t icase, const double* f, const double* g, const double* aux) {
    int rc = enter(h);
    if (rc != LBM_OK) return rc;
    if (check_case(h, icase) != LBM_OK) return LBM_ERR_INVALID_ARG;
    const int64_t n = (int64_t)h->prm[icase].nz * h->prm[icase].nr;
    double* df = h->state;
    double* dg = h->state + 9 * n;
    double* da = h->state + 18 * n;
    if (f) rc = cuda_ok(h, cudaMemcpyAsync(df, f, 9 * n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    if (rc == LBM_OK && g)
        rc = cuda_ok(h, cudaMemcpyAsync(dg, g, 9 * n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    if (rc == LBM_OK && aux)
        rc = cuda_ok(h, cudaMemcpyAsync(da, aux, 3 * n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    if (rc != LBM_OK) return rc;
    rc = cuda_ok(h, launch_set_state_any(h, icase, f ? df : nullptr, g ? dg : nullptr, aux ? da : nullptr));
    if (rc != LBM_OK) return rc;
    if (f) h->initialized[icase] = 1;
    return cuda_ok(h, cudaStreamSynchronize(h->stream));
}

int64_t lbm_checkpoint_size(const lbm_handle* h) {
    if (!h) return -1;
    const int64_t T = h->D.total;
    const int p = h->precision;
    return (int64_t)((T / 32) * block_bytes(p)) + 8 * (int64_t)h->ncases;
}

namespace {
// Copy the current state (the buffer of storage blocks the next step reads:
// populations, chi^{n-1}, p^{n-1}) to or from `buf` (host memory, or device
// memory when `device` is set).
int checkpoint_copy(lbm_sim* h, void* buf, bool save, bool device = false) {
    const int64_t T = h->D.total;
    const int p = h->precision;
    const int a = h->parity;
    struct Part {
        void* dev;
        size_t bytes;
    } parts[] = {{h->D.blk[a], (size_t)(T / 32) * block_bytes(p)}};
    char* cur = (char*)buf;
    for (const Part& q : parts) {
        const cudaMemcpyKind kind = device ? cudaMemcpyDeviceToDevice
                                           : (save ? cudaMemcpyDeviceToHost : cudaMemcpyHostToDevice);
        cudaError_t e = save ? cudaMemcpyAsync(cur, q.dev, q.bytes, kind, h->stream)
                             : cudaMemcpyAsync(q.dev, cur, q.bytes, kind, h->stream);
        if (e != cudaSuccess) return cuda_ok(h, e);
        cur += q.bytes;
    }
    if (!device) {
        if (save) std::memcpy(cur, h->case_steps.data(), 8 * h->ncases);
        else {
            std::memcpy(h->case_steps.data(), cur, 8 * h->ncases);
            for (int c = 0; c < h->ncases; ++c) h->initialized[c] = 1;
        }
    }
    return cuda_ok(h, cudaStreamSynchronize(h->stream));
}
}  // namespace

int lbm_checkpoint_save(lbm_handle* h, void* host_buf) {
    int rc = enter(h);
    if (rc != LBM_OK) return rc;
    if (!host_buf) return LBM_ERR_INVALID_ARG;
    return checkpoint_copy(h, host_buf, true);
}

int lbm_checkpoint_load(lbm_handle* h, const void* host_buf) {
    int rc = enter(h);
    if (rc != LBM_OK) return rc;
    if (!host_buf) return LBM_ERR_INVALID_ARG;
    return checkpoint_copy(h, const_cast<void*>(host_buf), false);
}

int32_t lbm_num_variants(void) { return kNumVariants; }

int lbm_set_variant(lbm_handle* h, int32_t variant) {
    int rc = enter(h);
    if (rc != LBM_OK) return rc;
    if (variant < 0 || variant >= kNumVariants) return LBM_ERR_INVALID_ARG;
    if (kVariantTMA[variant] && !h->tma_ok) return LBM_ERR_INVALID_ARG;
    h->variant = variant;
    return LBM_OK;
}

int lbm_autotune(lbm_handle* h, int32_t reps, int32_t* chosen) {
    int rc = enter(h);
    if (rc != LBM_OK) return rc;
    if (reps < 1) return LBM_ERR_INVALID_ARG;
    for (int c = 0; c < h->ncases; ++c)
        if (!h->initialized[c]) return LBM_ERR_STATE;
    const int64_t bytes = lbm_checkpoint_size(h);
    void* saved = nullptr;
    if (cudaMallocAsync(&saved, (size_t)bytes, h->stream) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ERR_OOM;
    }
    rc = checkpoint_copy(h, saved, true, true);
    if (rc != LBM_OK) {
        cudaFreeAsync(saved, h->stream);
        return rc;
    }
    const int parity0 = h->parity;
    const int64_t launches0 = h->launches;
    std::vector<int64_t> steps0 = h->case_steps;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return fail(h, LBM_ERR_CUDA);
    float best = 1e30f;
    int best_v = h->variant;
    for (int v = 0; v < kNumVariants && rc == LBM_OK; ++v) {
        if (kVariantTMA[v] && !h->tma_ok) continue;
        h->variant = v;
        rc = step_direct(h, 2);  // warm-up
        cudaEventRecord(e0, h->stream);
        if (rc == LBM_OK) rc = step_direct(h, 2 * reps);
        cudaEventRecord(e1, h->stream);
        if (rc == LBM_OK) rc = cuda_ok(h, cudaEventSynchronize(e1));
        float ms = 0.f;
        if (rc == LBM_OK) cudaEventElapsedTime(&ms, e0, e1);
        // a later candidate must be at least 1 % faster to replace an earlier
        // one, so near ties keep the earlier (default) launch shape
        if (rc == LBM_OK && ms < 0.99f * best) {
            best = ms;
            best_v = v;
        }
        h->parity = parity0;
        if (rc == LBM_OK) rc = checkpoint_copy(h, saved, false, true);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(saved, h->stream);
    h->variant = best_v;
    h->launches = launches0;
    h->case_steps = steps0;
    if (chosen) *chosen = best_v;
    return rc;
}

int64_t lbm_kernel_launches(const lbm_handle* h) { return h ? h->launches : 0; }

int lbm_destroy(lbm_handle* h) {
    if (!h) return LBM_OK;
    cudaSetDevice(h->device);
    release(h);
    delete h;
    return LBM_OK;
}

const char* lbm_strerror(int status) {
    switch (status) {
        case LBM_OK: return "ok";
        case LBM_ERR_INVALID_ARG: return "invalid argument";
        case LBM_ERR_CUDA: return "CUDA runtime error";
        case LBM_ERR_NONFINITE: return "non-finite value in phi, u or p";
        case LBM_ERR_TIMEOUT: return "bounded device wait timed out";
        case LBM_ERR_OOM: return "device out of memory";
        case LBM_ERR_STATE: return "call out of order (case not initialised)";
        default: return "unknown status";
    }
}

}  // extern "C"
