// lbm_device.cuh -- device-side arithmetic of one time step of the axisymmetric
// Allen-Cahn phase-field MRT lattice Boltzmann method (Liang et al., arXiv
// 1810.09299), written for sm_103a.
//
// The collision is done in moment space with the paper's closed forms:
// Eq. 21-23 (phase field) and Eq. 36-37 (hydrodynamics), the transform M of
// Sec. 2.2 unrolled into integer adds, M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6,
// 1/12, 1/6, 1/12, 1/4, 1/4).  Everything a node needs is recomputed from the
// populations each step: phi (Eq. 16) on a tile plus a two-node halo in shared
// memory, then the stencils (Eq. 39-40), the local macroscopic quantities and
// the collisions in registers, then the push streaming with the boundary rules.
#pragma once

#include <cuda.h>  // CUtensorMap (type only)
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cstddef>
#include <stdint.h>

#include "lbm_internal.h"

namespace axilbm {

// ---------------------------------------------------------------- lattice
// D2Q9 of Eq. 12 with c_i = (c_z, c_r): 0 (0,0), 1 (1,0), 2 (0,1), 3 (-1,0),
// 4 (0,-1), 5 (1,1), 6 (-1,1), 7 (-1,-1), 8 (1,-1).
__host__ __device__ constexpr int cz_of(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int cr_of(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__host__ __device__ constexpr double w_of(int i) {
    return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
}
__host__ __device__ constexpr int opp_of(int i) {
    return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 5 + 2) % 4) + 5);
}
// reflection r -> -r: 2 <-> 4, 5 <-> 8, 6 <-> 7
__host__ __device__ constexpr int rmir_of(int i) {
    return i == 2 ? 4 : i == 4 ? 2 : i == 5 ? 8 : i == 8 ? 5 : i == 6 ? 7 : i == 7 ? 6 : i;
}

// ---------------------------------------------------------------- per-case data
// Per-case constants in the arithmetic precision of the kernel (converted once
// on the host: the FP32 kernels never touch the FP64 pipe for parameters).
template <typename Real>
struct CaseReal {
    Real rho_l, rho_g, nu_l, nu_g, grav_z, n_eps;  // this order: node_macros reads the FP32
    Real beta, kappa, inv_W, mob;                  // block's first eight as two 16-byte loads
    Real sf[9];   // phase-field rates, derived entries already resolved (Eq. 18)
    Real sg[9];   // hydrodynamic rates; entries flagged in sg_local are 1/tau_g(x)
};
static_assert(offsetof(CaseReal<float>, nu_g) == 12 && offsetof(CaseReal<float>, grav_z) == 16 &&
                  offsetof(CaseReal<float>, kappa) == 28,
              "FP32 parameter order read by node_macros");

// Case c owns the handle's nodes [off, off + plane): node (k, j) is node
// off + k * pitch + j (pitch = nr rounded up to 32, off a multiple of 32).
// How nodes are stored is described with Block below.  Node indices inside a
// case are 32-bit.
struct CaseDev {
    int32_t nr, nz, pitch, zper;
    int32_t p_coupling;
    uint32_t sg_local;  // bit i set: sg[i] = 1/tau_g(x) from the local viscosity (Eq. 34)
    int64_t off;        // node offset of the case (see above)
    int32_t plane;      // nz * pitch
    int32_t collision;  // 0: orthogonal moments (M, Sec. 2.2); 1: raw moments (see raw_from_ortho)
    int64_t dense_off;  // first node of the case in the dense concatenation of every case's [nz][nr]
    // the FP32 parameters first, 16-byte aligned (measured -0.45 % on the
    // mixed FP16 step against the FP64 block first; FP32 unchanged)
    CaseReal<float> pf;
    CaseReal<double> pd;
};
static_assert(sizeof(CaseDev) % 16 == 0, "CaseDev is copied to shared memory by a bulk copy");
static_assert(offsetof(CaseDev, pf) % 16 == 0 && offsetof(CaseDev, pd) % 8 == 0, "parameter block alignment");

template <typename Real>
__device__ __forceinline__ const CaseReal<Real>& case_params(const CaseDev& C);
template <>
__device__ __forceinline__ const CaseReal<double>& case_params<double>(const CaseDev& C) { return C.pd; }
template <>
__device__ __forceinline__ const CaseReal<float>& case_params<float>(const CaseDev& C) { return C.pf; }

// One tile of one case: (case, k0, j0)
struct TileDev {
    int32_t c, k0, j0, pad;
};

// The same tile with its case's geometry: the case's first storage block
// (blk0 = off / 32), one z row in blocks (pitch / 32), nr, nz and the z
// periodicity.  A step variant's tile list is followed in device memory by one
// of these per tile, so that a kernel can address the tile's nodes and its phi
// ring as soon as this record arrives, before the case record.
struct TileGeo {
    int32_t c, k0, j0, blk0;
    int32_t rowblk, nr, nz, zper;
};

// ---------------------------------------------------------------- storage codecs
// Populations are stored as PT (f_1..8, g_0..8) and F0T (f_0).  wr = w_i * r of
// the node the value is stored at (known to writer and reader), inv_wr = 1/wr.
//
// In the FP32 and 16-bit codecs f_0 is the node's mass ledger, a double-float
// pair (hi, lo): each step it is rewritten as (sum of the node's incoming
// populations) minus (its outgoing f_1..8), accumulated with error-free
// TwoSum steps (Knuth), so the sum of all populations is conserved to ~2^-48
// relative although the collision runs in FP32 and f_1..8 are rounded.
struct FF {
    float hi, lo;
};
__device__ __forceinline__ void ff_add(FF& a, float x) {
    const float s = a.hi + x;
    const float bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (x - bb);
    a.hi = s;
    a.lo += e;
}
__device__ __forceinline__ FF ff_norm(FF a) {
    const float h = a.hi + a.lo;
    return FF{h, a.lo - (h - a.hi)};
}

struct CodecF64 {
    using Real = double;
    using PT = double;
    using F0T = double;
    static constexpr bool kLedger = false;
    static constexpr bool kExactLedger = false;
    static constexpr bool kGrid = false;
    static constexpr bool kStreamStores = false;
    using PT2 = double2;  // (f_i, g_i) of one direction, stored together
    __device__ static Real dec_f(PT v, Real) { return v; }
    __device__ static PT enc_f(Real v, Real, Real) { return v; }
    __device__ static Real dec_g(PT v, Real) { return v; }
    __device__ static PT enc_g(Real v, Real, Real) { return v; }
    __device__ static PT2 enc_pair(Real f, Real g, Real, Real) { return make_double2(f, g); }
};

struct CodecF32 {
    using Real = float;
    using PT = float;
    using F0T = float2;
    using PT2 = float2;
    static constexpr bool kLedger = true;
    static constexpr bool kExactLedger = false;
    static constexpr bool kGrid = false;
    static constexpr bool kStreamStores = false;
    __device__ static Real dec_f(PT v, Real) { return v; }
    __device__ static PT enc_f(Real v, Real, Real) { return v; }
    __device__ static Real dec_g(PT v, Real) { return v; }
    __device__ static PT enc_g(Real v, Real, Real) { return v; }
    __device__ static PT2 enc_pair(Real f, Real g, Real, Real) { return make_float2(f, g); }
};

// Mixed-precision adds and FMAs (PTX ISA 8.6, sm_100 family): the 16-bit
// operands are taken exactly and the FP32 result is rounded once, in one
// instruction (the add checked bit for bit against a conversion followed by
// an FP32 add over every FP16 value on the GPU).
__device__ __forceinline__ float add_h(__half h, float c) {
    float d;
    asm("add.rn.f32.f16 %0, %1, %2;" : "=f"(d) : "h"(__half_as_ushort(h)), "f"(c));
    return d;
}
__device__ __forceinline__ float add_h(__nv_bfloat16 h, float c) {
    float d;
    asm("add.rn.f32.bf16 %0, %1, %2;" : "=f"(d) : "h"(__bfloat16_as_ushort(h)), "f"(c));
    return d;
}
// a * b + c with a, b 16-bit (b given by its bits)
__device__ __forceinline__ float fma_h(__half a, uint16_t b, float c) {
    float d;
    asm("fma.rn.f32.f16 %0, %1, %2, %3;" : "=f"(d) : "h"(__half_as_ushort(a)), "h"(b), "f"(c));
    return d;
}
__device__ __forceinline__ float fma_h(__nv_bfloat16 a, uint16_t b, float c) {
    float d;
    asm("fma.rn.f32.bf16 %0, %1, %2, %3;" : "=f"(d) : "h"(__bfloat16_as_ushort(a)), "h"(b), "f"(c));
    return d;
}

// kStreamStores: the step writes its pushed populations with evict-first
// stores (measured: -1.5 % on the 16-bit step, +2.8 % on the FP32 one).
//
// FP16 storage on a grid.  Column j (r = j + 1/2) has the scales S_i of its
// directions: S_a = w_1 r = r / 9 rounded up to kScaleBits significant bits,
// S_i = S_a for i = 1..4, S_a / 4 for i = 5..8, 4 S_a for i = 0 (the weights'
// ratios), so S_i = w_i r / alpha with alpha in (2/3, 1] at 2 bits.  f_i
// (i = 1..8) is stored as the centred deviation
//   h_i = f_i / S_i - 1/2,
// first rounded to a multiple of 2^-kGridExp, then to the 16-bit format
// (which keeps it on that grid), and decoded as
//   f_i = (h_i + 1/2) S_i   (one mixed-precision FMA),
// which is exact: a number of kGridExp + 1 bits times one of kScaleBits bits,
// kGridExp + kScaleBits <= 16.  f_i = 0 (the phase phi = 0) is stored as
// exactly -1/2.  Every value a node's mass ledger adds or subtracts (its
// incoming f_1..8 decoded at its own column, the f_1..8 it stores decoded at
// the destination columns j-1, j, j+1, and its own f_0) is then a multiple of
// q = 2^-kGridExp ulp(S_5 of column max(j - 1, 0)), ulp at kScaleBits bits,
// and every partial sum (at most about r phi) stays below 2^24 q for phi up to
// about 2, so plain FP32 additions of them are exact: f_0 is one FP32 value,
// (sum of the incoming populations) minus (the stored outgoing f_1..8), and the
// step conserves the sum of all populations exactly.
// g_i is stored as kGScale g_i / S_i (the scale keeps typical values out of
// FP16's subnormal range).
__device__ __forceinline__ uint16_t bits16(__half v) { return __half_as_ushort(v); }
__device__ __forceinline__ uint16_t bits16(__nv_bfloat16 v) { return __bfloat16_as_ushort(v); }
template <typename PT>
__device__ __forceinline__ PT to16(float v);
template <>
__device__ __forceinline__ __half to16<__half>(float v) { return __float2half_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 to16<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// The constants of one column (see above).  Axis class (directions 1..4),
// diagonal class (5..8); S16: S of both classes as 16-bit numbers (axis low),
// S16g: the g decode scales S / kGScale of both classes, S16g0: that of g_0.
struct GridCol {
    float invS_a, G_a, cS_a, S_a;  // 1 / S, kGScale / S, S / 2, S
    float invS_d, G_d, cS_d, S_d;
    uint32_t S16, S16g, S16g0, pad;
};

// S_a of column j
template <class Codec>
__device__ __forceinline__ float grid_sa(int j) {
    constexpr uint32_t mask = (1u << (24 - Codec::kScaleBits)) - 1u;  // 0 at 24 bits
    const uint32_t u = __float_as_uint(__fmul_rn((float)j + 0.5f, 1.0f / 9.0f));
    return __uint_as_float((u + mask) & ~mask);
}

template <class Codec>
__device__ __forceinline__ GridCol grid_col(int j) {
    using PT = typename Codec::PT;
    constexpr float gs = Codec::kGScale;
    const float Sa = grid_sa<Codec>(j), Sd = 0.25f * Sa, S0 = 4.0f * Sa;
    const float inv = __frcp_rn(Sa);
    GridCol g;
    g.invS_a = inv;
    g.invS_d = 4.0f * inv;
    g.G_a = gs * inv;
    g.G_d = gs * g.invS_d;
    g.cS_a = 0.5f * Sa;
    g.cS_d = 0.5f * Sd;
    g.S_a = Sa;
    g.S_d = Sd;
    g.S16 = (uint32_t)bits16(to16<PT>(Sa)) | ((uint32_t)bits16(to16<PT>(Sd)) << 16);
    g.S16g = (uint32_t)bits16(to16<PT>(Sa / gs)) | ((uint32_t)bits16(to16<PT>(Sd / gs)) << 16);
    g.S16g0 = (uint32_t)bits16(to16<PT>(S0 / gs));
    g.pad = 0u;
    return g;
}

// Rounding of a 16-bit-storage f_0 onto the ledger grid of column j: the
// multiple of q = 2^-kGridExp ulp(S_5(max(j - 1, 0))) nearest to x (x + 1.5 *
// 2^23 q - 1.5 * 2^23 q, for |x| < 2^22 q).
template <class Codec>
__device__ __forceinline__ float grid_round_f0(float x, int j) {
    const uint32_t ex = (__float_as_uint(0.25f * grid_sa<Codec>(max(j - 1, 0))) >> 23) & 0xffu;
    const float m = __uint_as_float(((ex + 24u - Codec::kScaleBits - Codec::kGridExp) << 23) | 0x400000u);
    return __fadd_rn(__fadd_rn(x, m), -m);
}

template <class PT_, class PT2_, int kGS, int kE, int kBits>
struct CodecGrid16 {
    using Real = float;
    using PT = PT_;
    using F0T = float;
    using PT2 = PT2_;
    static constexpr bool kLedger = false;
    static constexpr bool kExactLedger = true;  // one FP32 word, exact sums on the grid
    static constexpr bool kGrid = true;         // column constants (GridCol)
    static constexpr bool kStreamStores = true;
    static constexpr float kGScale = (float)kGS;
    static constexpr int kGridExp = kE, kScaleBits = kBits;
    static_assert(kE + kBits <= 16, "ledger sums of at most 24 bits");
    // x + kMagic - kMagic rounds |x| < 2^(22 - kE) to a multiple of 2^-kE
    static constexpr float kMagic = 1.5f * (float)(1 << (23 - kE));
    // D: the diagonal class (directions 5..8), else the axis class (1..4); a
    // constant wherever it is called (unrolled direction loops)
    // f_i from its stored value at the column of g
    __device__ static float dec_f(PT h, const GridCol& g, bool D) {
        return fma_h(h, (uint16_t)(D ? g.S16 >> 16 : g.S16 & 0xffffu), D ? g.cS_d : g.cS_a);
    }
    __device__ static float dec_g(PT h, const GridCol& g, bool D) {
        return fma_h(h, (uint16_t)(D ? g.S16g >> 16 : g.S16g & 0xffffu), 0.0f);
    }
    __device__ static float dec_g0(PT h, const GridCol& g) { return fma_h(h, (uint16_t)g.S16g0, 0.0f); }
    // the stored h of f: f / S - 1/2 on the 2^-kE grid
    __device__ static float grid_h(float f, const GridCol& g, bool D) {
        return __fadd_rn(__fmaf_rn(f, D ? g.invS_d : g.invS_a, kMagic - 0.5f), -kMagic);
    }
    // f and g of a direction as one stored pair (a packed FMA and add for
    // both, bit-identical, measured 1.5 % slower in the packed two-node step)
    __device__ static PT2 enc_pair(float f, float gv, const GridCol& g, bool D) {
        PT2 e;
        e.x = to16<PT>(grid_h(f, g, D));
        e.y = to16<PT>(gv * (D ? g.G_d : g.G_a));
        return e;
    }
    __device__ static PT enc_f(float f, const GridCol& g, bool D) { return to16<PT>(grid_h(f, g, D)); }
    __device__ static PT enc_g(float gv, const GridCol& g, bool D) { return to16<PT>(gv * (D ? g.G_d : g.G_a)); }
    // g_0 (S_0 = 4 S_a)
    __device__ static PT enc_g0(float gv, const GridCol& g) { return to16<PT>(gv * (0.25f * g.G_a)); }
};
// (kGridExp, kScaleBits) of FP16, measured on the 64 x 128 static drop
// against the FP64 oracle (2000 steps, phi max / L2; paper's collision, then
// the raw-moment one): (12, 4) 3.4e-2 / 7.2e-4; (13, 3) 4.0e-2 / 8.3e-4 and
// 4.8e-2 / 1.0e-3; (14, 2) 1.7e-2 / 3.5e-4 and 2.0e-2 / 4.3e-4; (15, 1)
// 2.4e-2 / 5.1e-4 and 7.1e-3 / 1.6e-4.  (14, 2) is the one within both
// collisions' bounds.
#ifndef AXILBM_H16_E
#define AXILBM_H16_E 14
#define AXILBM_H16_B 2
#endif
using CodecH16 = CodecGrid16<__half, __half2, 256, AXILBM_H16_E, AXILBM_H16_B>;

// bfloat16 storage keeps the centred deviation on the full FP32 scale w_i r:
// f_i / (w_i r) - 1/2 and g_i / (w_i r), decoded as h wr + wr/2 in one
// explicit FMA (wr/2 is exact), the same expression for the writer's mass
// ledger and for the next reader, so both round alike; f_0 is the
// double-float ledger of the FP32 codec.  bfloat16 keeps 8 significant bits,
// so any scale short enough for the grid's exact decode leaves alpha = w r / S
// a few of its units off 1, and a column's liquid deviations all round the
// same way.  On grids of (9, 7), (10, 6) and (11, 5) bits the 256 x 1024
// rising bubble at ratio 1000 went non-finite between 17,500 and 25,000
// steps; this form follows it through 25,000 steps.
struct CodecB16 {
    using Real = float;
    using PT = __nv_bfloat16;
    using F0T = float2;
    using PT2 = __nv_bfloat162;
    static constexpr bool kLedger = true;
    static constexpr bool kExactLedger = false;
    static constexpr bool kGrid = false;
    static constexpr bool kStreamStores = true;
    __device__ static Real dec_f(PT v, Real wr) { return __fmaf_rn(__bfloat162float(v), wr, 0.5f * wr); }
    __device__ static PT enc_f(Real v, Real, Real inv_wr) { return __float2bfloat16_rn(v * inv_wr - 0.5f); }
    __device__ static Real dec_g(PT v, Real wr) { return __bfloat162float(v) * wr; }
    __device__ static PT enc_g(Real v, Real, Real inv_wr) { return __float2bfloat16_rn(v * inv_wr); }
    __device__ static PT2 enc_pair(Real f, Real g, Real, Real inv_wr) {
        return __floats2bfloat162_rn(f * inv_wr - 0.5f, g * inv_wr);
    }
};

// phi of a bfloat16 node (Eq. 16) from its raw stored f_0 and f_1..8: with
// the decode f_i = (h_i + 1/2) w_i r the sum f_i / r reads
//   phi = f_0 / r + (h_1 + .. + h_4 + 2) / 9 + (h_5 + .. + h_8 + 2) / 36,
// summed from the stored values with eight mixed-precision adds (no decode);
// every path that forms phi of such a node uses this one form.
template <typename PT>
__device__ __forceinline__ float phi_from_halves(float f0, const PT* h, float inv_r) {
    float a = 2.0f, b = 2.0f;
#pragma unroll
    for (int i = 0; i < 4; ++i) a = add_h(h[i], a);
#pragma unroll
    for (int i = 4; i < 8; ++i) b = add_h(h[i], b);
    return __fmaf_rn(f0, inv_r, __fmaf_rn(a, 1.0f / 9.0f, b * (1.0f / 36.0f)));
}

// phi of a 16-bit node (Eq. 16) from its stored f_0 and h_1..8:
//   sum f_i / r = (f_0 + S_a (A + B / 4)) / r,  A = 2 + h_1 + .. + h_4,
//   B = 2 + h_5 + .. + h_8,
// summed from the stored values with eight mixed-precision adds (no decode);
// every path that forms phi of a 16-bit node uses this one form, so the phi
// window is the same whichever tile or launch shape computes a cell.
template <typename PT>
__device__ __forceinline__ float phi_grid(float f0, const PT* h, float inv_r, float Sa) {
    float a = 2.0f, b = 2.0f;
#pragma unroll
    for (int i = 0; i < 4; ++i) a = add_h(h[i], a);
#pragma unroll
    for (int i = 4; i < 8; ++i) b = add_h(h[i], b);
    return __fmul_rn(__fmaf_rn(Sa, __fmaf_rn(b, 0.25f, a), f0), inv_r);
}

// f_0 as a value of the arithmetic type.
__device__ __forceinline__ double f0_value(double v) { return v; }
__device__ __forceinline__ float f0_value(float2 v) { return v.x + v.y; }
__device__ __forceinline__ float f0_value(float v) { return v; }

// ---------------------------------------------------------------- storage layout
// Nodes are stored in groups of 32 consecutive nodes of one row: node L of
// the handle lies in group L / 32 at lane L % 32.  Each group owns one block
// per state buffer holding every stored value of its 32 nodes,
//   f_0 [32 x F0T] | (f_i, g_i) for i = 1..8 [8][32 x 2 PT] | g_0 [32 x PT] |
//   (chi_z, chi_r) [32 x 2 Real] | p [32 x Real],
// padded to a multiple of 128 bytes.  f_i and g_i of a direction are always
// pushed to the same neighbour, so they are stored side by side and move as
// one vector access.  A warp reads or writes one slot of its 32 nodes as one
// contiguous run, and all runs of a node group lie together in memory, so the
// step's streams per node share DRAM pages and translation entries (a pure
// data-movement test of the step's traffic moved 13 % more bytes per second
// this way than with one plane per array).  chi and p live in both buffers:
// the step reads them from the buffer it reads and writes them to the buffer
// it writes.
template <class Codec>
struct Block {
    using PT = typename Codec::PT;
    using F0T = typename Codec::F0T;
    using Real = typename Codec::Real;
    static constexpr int off_f0 = 0;
    static constexpr int off_pairs = 32 * (int)sizeof(F0T);
    static constexpr int pair_slot = 32 * 2 * (int)sizeof(PT);  // bytes of one direction's pair slot
    static constexpr int off_g0 = off_pairs + 8 * pair_slot;
    static constexpr int off_chi = off_g0 + 32 * (int)sizeof(PT);
    static constexpr int off_p = off_chi + 32 * 2 * (int)sizeof(Real);
    static constexpr int bytes = block_bytes_of((int)sizeof(F0T), (int)sizeof(PT), (int)sizeof(Real));
    static_assert(off_p + 32 * (int)sizeof(Real) <= bytes, "block layout");
    static_assert(sizeof(typename Codec::PT2) == 2 * sizeof(PT), "pair type");
};

// One node's values in one buffer: its group's block and its lane.
template <class Codec>
struct Node {
    using PT = typename Codec::PT;
    using PT2 = typename Codec::PT2;
    using F0T = typename Codec::F0T;
    using Real = typename Codec::Real;
    using L = Block<Codec>;
    unsigned char* blk;
    int lane;
    __device__ __forceinline__ F0T& f0() const { return reinterpret_cast<F0T*>(blk + L::off_f0)[lane]; }
    // the (f_i, g_i) pair of direction i = 1..8
    __device__ __forceinline__ PT2& pair(int i) const {
        return reinterpret_cast<PT2*>(blk + L::off_pairs + (i - 1) * L::pair_slot)[lane];
    }
    __device__ __forceinline__ PT& f(int i) const {
        return reinterpret_cast<PT*>(blk + L::off_pairs + (i - 1) * L::pair_slot)[2 * lane];
    }
    __device__ __forceinline__ PT& g(int i) const {
        return i == 0 ? reinterpret_cast<PT*>(blk + L::off_g0)[lane]
                      : reinterpret_cast<PT*>(blk + L::off_pairs + (i - 1) * L::pair_slot)[2 * lane + 1];
    }
    __device__ __forceinline__ Real& chz() const { return reinterpret_cast<Real*>(blk + L::off_chi)[2 * lane]; }
    __device__ __forceinline__ Real& chr() const { return reinterpret_cast<Real*>(blk + L::off_chi)[2 * lane + 1]; }
    __device__ __forceinline__ Real& p() const { return reinterpret_cast<Real*>(blk + L::off_p)[lane]; }
};

// A node's direction pairs addressed by one byte pointer (block + lane *
// sizeof(PT2)): the pair of every direction i = 1..8 is that pointer plus a
// constant.
template <class Codec>
struct PtRef {
    using PT2 = typename Codec::PT2;
    using L = Block<Codec>;
    unsigned char* q;
    __device__ __forceinline__ PT2& pair(int i) const {
        return *reinterpret_cast<PT2*>(q + L::off_pairs + (i - 1) * L::pair_slot);
    }
};

// The two state buffers (arrays of blocks) of one step.
template <class Codec>
struct StateDev {
    const unsigned char* in;  // the buffer the step reads
    unsigned char* out;       // the buffer it writes
};

// The buffers of one case; nodes are addressed by loc = k * pitch + j.
template <class Codec>
struct CaseView {
    unsigned char* in;   // block of the case's first group in the buffer read
    unsigned char* out;  // ... in the buffer written
    int pitch;
    __device__ __forceinline__ Node<Codec> in_node(int loc) const {
        return Node<Codec>{in + (int64_t)(loc >> 5) * Block<Codec>::bytes, loc & 31};
    }
    __device__ __forceinline__ Node<Codec> out_node(int loc) const {
        return Node<Codec>{out + (int64_t)(loc >> 5) * Block<Codec>::bytes, loc & 31};
    }
    __device__ __forceinline__ PtRef<Codec> out_pt(int loc) const {
        return PtRef<Codec>{out + (int64_t)(loc >> 5) * Block<Codec>::bytes +
                            (loc & 31) * (int)sizeof(typename Codec::PT2)};
    }
};

template <class Codec>
__device__ __forceinline__ CaseView<Codec> case_view(const StateDev<Codec>& S, const CaseDev& C) {
    CaseView<Codec> v;
    const int64_t b0 = (C.off >> 5) * Block<Codec>::bytes;
    v.in = const_cast<unsigned char*>(S.in) + b0;
    v.out = S.out + b0;
    v.pitch = C.pitch;
    return v;
}

// ---------------------------------------------------------------- ghost rules
// Sec. 2.3: mirror about the axis (r = 0 lies between j = -1 and j = 0), mirror
// about the halfway wall planes, periodic wrap in z.  The result is clamped
// into the domain so that halo cells beyond the two-node ghost ring (ragged
// tiles) stay in bounds; they are never used by a real node.
__device__ __forceinline__ int ghost_r(int j, int nr) {
    if (j < 0) j = -1 - j;
    if (j >= nr) j = 2 * nr - 1 - j;
    return min(max(j, 0), nr - 1);
}
__device__ __forceinline__ int ghost_z(int k, int nz, int zper) {
    if (zper) {
        k %= nz;
        if (k < 0) k += nz;
        return k;
    }
    if (k < 0) k = -1 - k;
    if (k >= nz) k = 2 * nz - 1 - k;
    return min(max(k, 0), nz - 1);
}

// phi of a node from its raw stored f_0 (F0T) and f_1..8 (Eq. 16): the
// plain sum in FP64 and FP32 storage, phi_grid in FP16 storage (Sa: S_a of
// the node's column; unused otherwise), phi_from_halves in bfloat16 storage.
template <class Codec>
__device__ __forceinline__ typename Codec::Real phi_of(const typename Codec::F0T& f0raw,
                                                        const typename Codec::PT* fraw,
                                                        typename Codec::Real inv_r, float Sa = 0.0f) {
    using Real = typename Codec::Real;
    if constexpr (Codec::kGrid) {
        return phi_grid(f0_value(f0raw), fraw, inv_r, Sa);
    } else if constexpr (sizeof(typename Codec::PT) == 2) {
        return phi_from_halves(f0_value(f0raw), fraw, inv_r);
    } else {
        Real s = (Real)f0_value(f0raw);
#pragma unroll
        for (int i = 0; i < 8; ++i) s += fraw[i];
        return s * inv_r;
    }
}

// The stored f_0 and f_1..8 of node n, the values phi is summed from (Eq. 16):
// loaded ahead of their use, then phi_of(f0, f, 1 / r, S_a) gives what
// node_phi gives.
template <class Codec>
__device__ __forceinline__ void load_phi_raw(const Node<Codec>& n, typename Codec::F0T& f0,
                                             typename Codec::PT* f) {
    f0 = n.f0();
#pragma unroll
    for (int i = 1; i < 9; ++i) f[i - 1] = n.f(i);
}

// phi at an in-domain node from its stored populations (Eq. 16).  FP64 and
// FP32: each load feeds the running sum (the order phi_of sums in).
template <class Codec>
__device__ __forceinline__ typename Codec::Real node_phi(const Node<Codec>& n, typename Codec::Real inv_r,
                                                          float Sa = 0.0f) {
    using Real = typename Codec::Real;
    if constexpr (sizeof(typename Codec::PT) == 2) {
        typename Codec::PT fraw[8];
#pragma unroll
        for (int i = 1; i < 9; ++i) fraw[i - 1] = n.f(i);
        return phi_of<Codec>(n.f0(), fraw, inv_r, Sa);
    } else {
        Real s = (Real)f0_value(n.f0());
#pragma unroll
        for (int i = 1; i < 9; ++i) s += n.f(i);
        return s * inv_r;
    }
}
// ---------------------------------------------------------------- arithmetic helpers
// FP32: the hardware approximate reciprocal, division and square root (a few
// ulp, far below the FP32 rounding the method accumulates over a run), with
// subnormal inputs and results flushed to zero (PTX .approx.ftz): values
// below 2^-126 arise only in the far field at rest, and the forms that keep
// them cost 1.7 % (FP32) to 3.5 % (16-bit storage) of the step;
// FP64: IEEE division and square root, as in the oracle.
__device__ __forceinline__ float rcp_(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ double rcp_(double x) { return 1.0 / x; }
__device__ __forceinline__ float div_(float a, float b) {
    float y;
    asm("div.approx.ftz.f32 %0, %1, %2;" : "=f"(y) : "f"(a), "f"(b));
    return y;
}
__device__ __forceinline__ double div_(double a, double b) { return a / b; }
__device__ __forceinline__ float sqrt_(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }

// ---------------------------------------------------------------- macroscopic part
template <typename Real>
struct Macro {
    Real r, inv_r, phi, rho, nu;
    Real gz, gr, lap;
    Real uz, ur, p, pstar;
    Real Fz, Fr;
    Real nzn, nrn, lam;
    Real sg[9];
    Real mg[9];  // M g (hydrodynamic moments before collision)
};

// Stencils (Eq. 39, Eq. 40) from the shared phi window centred on (a, b).
// With x1, x2 the values one and two links along c_i, d_i = 8 x1 - x2 and
// u_i = 16 x1 - x2:
//   grad phi = sum_i w_i c_i d_i / (6 cs^2),
//   lap phi  = (sum_i w_i u_i - 15 phi sum_i w_i) / (6 cs^2),
// with 6 cs^2 = 2 and sum_{i>0} w_i = 5/9, the sums grouped by weight class.
template <typename Real, int LD>
__device__ __forceinline__ void stencil(const Real* sphi, int a, int b, Real& gz, Real& gr, Real& lap) {
    const Real c0 = sphi[a * LD + b];
    Real d[9], u[9];
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const Real x1 = sphi[(a + cz_of(i)) * LD + (b + cr_of(i))];
        const Real x2 = sphi[(a + 2 * cz_of(i)) * LD + (b + 2 * cr_of(i))];
        d[i] = (Real)8 * x1 - x2;
        u[i] = (Real)8 * x1 + d[i];
    }
    const Real h1 = (Real)(1.0 / 18.0), h2 = (Real)(1.0 / 72.0);  // w_i / 2 on the axes and diagonals
    gz = h1 * (d[1] - d[3]) + h2 * ((d[5] + d[8]) - (d[6] + d[7]));
    gr = h1 * (d[2] - d[4]) + h2 * ((d[5] + d[6]) - (d[7] + d[8]));
    lap = h1 * ((u[1] + u[2]) + (u[3] + u[4])) + h2 * ((u[5] + u[6]) + (u[7] + u[8])) - (Real)(25.0 / 6.0) * c0;
}

// M g for the nine hydrodynamic populations (rows of M in Sec. 2.2).
template <typename Real>
__device__ __forceinline__ void moments(const Real* x, Real* m) {
    const Real a14 = x[1] + x[2] + x[3] + x[4];
    const Real a58 = x[5] + x[6] + x[7] + x[8];
    m[0] = x[0] + a14 + a58;
    m[1] = (Real)-4 * x[0] - a14 + (Real)2 * a58;
    m[2] = (Real)4 * x[0] - (Real)2 * a14 + a58;
    const Real d57 = x[5] - x[7], d68 = x[6] - x[8];
    m[3] = x[1] - x[3] + d57 - d68;
    m[4] = (Real)-2 * (x[1] - x[3]) + d57 - d68;
    m[5] = x[2] - x[4] + d57 + d68;
    m[6] = (Real)-2 * (x[2] - x[4]) + d57 + d68;
    m[7] = x[1] - x[2] + x[3] - x[4];
    m[8] = x[5] - x[6] + x[7] - x[8];
}

// x = M^-1 m with M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4).
template <typename Real>
__device__ __forceinline__ void inverse_moments(const Real* m, Real* x) {
    const Real a0 = m[0] * (Real)(1.0 / 9.0);
    const Real a1 = m[1] * (Real)(1.0 / 36.0);
    const Real a2 = m[2] * (Real)(1.0 / 36.0);
    const Real a3 = m[3] * (Real)(1.0 / 6.0);
    const Real a4 = m[4] * (Real)(1.0 / 12.0);
    const Real a5 = m[5] * (Real)(1.0 / 6.0);
    const Real a6 = m[6] * (Real)(1.0 / 12.0);
    const Real a7 = m[7] * (Real)0.25;
    const Real a8 = m[8] * (Real)0.25;
    const Real e = a0 - a1 - (Real)2 * a2;   // axis directions, isotropic part
    const Real d = a0 + (Real)2 * a1 + a2;   // diagonal directions, isotropic part
    const Real jz = a3 - (Real)2 * a4, jr = a5 - (Real)2 * a6;
    const Real qz = a3 + a4, qr = a5 + a6;
    x[0] = a0 - (Real)4 * a1 + (Real)4 * a2;
    x[1] = e + jz + a7;
    x[2] = e + jr - a7;
    x[3] = e - jz + a7;
    x[4] = e - jr - a7;
    x[5] = d + qz + qr + a8;
    x[6] = d - qz + qr - a8;
    x[7] = d - qz - qr + a8;
    x[8] = d + qz - qr - a8;
}

// ---------------------------------------------------------------- raw moments
// The non-orthogonal basis of the raw-moment collision (the extension named
// in Sec. 4): k_0..8 = sums of x_i times 1, c_z, c_r, c_z^2 + c_r^2,
// c_z^2 - c_r^2, c_z c_r, c_z^2 c_r, c_z c_r^2, c_z^2 c_r^2.  On D2Q9 each is a
// fixed combination of the orthogonal moments of M (c^2 = (e + 4) / 3,
// c_z c_r^2 = (q_z + 2 j_z) / 3, c_z^2 c_r^2 = (eps + 2 e + 4) / 9, ...), so
// the collision stays in the orthogonal moments the step already has and maps
// the deviations into the raw basis and back.
template <typename Real>
__device__ __forceinline__ void raw_from_ortho(const Real* m, Real* k) {
    k[0] = m[0];
    k[1] = m[3];
    k[2] = m[5];
    k[3] = (m[1] + (Real)4 * m[0]) * (Real)(1.0 / 3.0);
    k[4] = m[7];
    k[5] = m[8];
    k[6] = (m[6] + (Real)2 * m[5]) * (Real)(1.0 / 3.0);
    k[7] = (m[4] + (Real)2 * m[3]) * (Real)(1.0 / 3.0);
    k[8] = (m[2] + (Real)2 * m[1] + (Real)4 * m[0]) * (Real)(1.0 / 9.0);
}
template <typename Real>
__device__ __forceinline__ void ortho_from_raw(const Real* k, Real* m) {
    m[0] = k[0];
    m[3] = k[1];
    m[5] = k[2];
    m[1] = (Real)3 * k[3] - (Real)4 * k[0];
    m[7] = k[4];
    m[8] = k[5];
    m[6] = (Real)3 * k[6] - (Real)2 * k[2];
    m[4] = (Real)3 * k[7] - (Real)2 * k[1];
    m[2] = (Real)9 * k[8] - (Real)6 * k[3] + (Real)4 * k[0];
}
// m+ = m - A^-1 S A (m - meq) + A^-1 (I - S/2) A src, A = raw_from_ortho: the
// collision of Eq. 10 / Eq. 24 with S the rates of the raw moments.
template <typename Real>
__device__ __forceinline__ void raw_relax(const Real* m, const Real* meq, const Real* src, const Real* s, Real* mp) {
    Real d[9], dk[9], sk[9], dm[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) d[i] = m[i] - meq[i];
    raw_from_ortho(d, dk);
    raw_from_ortho(src, sk);
#pragma unroll
    for (int i = 0; i < 9; ++i) dk[i] = -s[i] * dk[i] + ((Real)1 - (Real)0.5 * s[i]) * sk[i];
    ortho_from_raw(dk, dm);
#pragma unroll
    for (int i = 0; i < 9; ++i) mp[i] = m[i] + dm[i];
}

// ---------------------------------------------------------------- paired FP32 transforms
// The two LBEs apply the same moment matrix to their nine populations.  In
// FP32 the pair (f_i, g_i) is held as one float2 and transformed with the
// packed FP32x2 instructions of sm_100-family GPUs (one instruction per pair,
// IEEE round-to-nearest per component); a - b is the exact FMA b * -1 + a.
__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ float2 p_fma(float s, float2 a, float2 b) { return __ffma2_rn(make_float2(s, s), a, b); }
__device__ __forceinline__ float2 p_mul(float s, float2 a) { return __fmul2_rn(make_float2(s, s), a); }

// Two double-float accumulators advanced together: the error-free TwoSum
// steps of ff_add, one packed instruction per step for both lanes.
struct FF2 {
    float2 hi, lo;
};
__device__ __forceinline__ void ff2_add(FF2& a, float2 x) {
    const float2 s = p_add(a.hi, x);
    const float2 bb = p_sub(s, a.hi);
    const float2 e = p_add(p_sub(a.hi, p_sub(s, bb)), p_sub(x, bb));
    a.hi = s;
    a.lo = p_add(a.lo, e);
}
// a -= x (TwoSum of a.hi and -x)
__device__ __forceinline__ void ff2_sub(FF2& a, float2 x) {
    const float2 s = p_sub(a.hi, x);
    const float2 bb = p_sub(s, a.hi);
    const float2 e = p_sub(p_sub(a.hi, p_sub(s, bb)), p_add(x, bb));
    a.hi = s;
    a.lo = p_add(a.lo, e);
}
// The sum of both lanes as one normalised double-float.
__device__ __forceinline__ FF ff2_merge(const FF2& a) {
    FF r{a.hi.x, a.lo.x + a.lo.y};
    ff_add(r, a.hi.y);
    return ff_norm(r);
}

// M x for a pair of population sets (the rows of moments()).
__device__ __forceinline__ void moments_p(const float2* x, float2* m) {
    const float2 s13 = p_add(x[1], x[3]), s24 = p_add(x[2], x[4]);
    const float2 s57 = p_add(x[5], x[7]), s68 = p_add(x[6], x[8]);
    const float2 a14 = p_add(s13, s24), a58 = p_add(s57, s68);
    m[0] = p_add(p_add(x[0], a14), a58);
    m[1] = p_fma(-4.0f, x[0], p_sub(p_add(a58, a58), a14));
    m[2] = p_fma(4.0f, x[0], p_fma(-2.0f, a14, a58));
    const float2 d13 = p_sub(x[1], x[3]), d24 = p_sub(x[2], x[4]);
    const float2 d57 = p_sub(x[5], x[7]), d68 = p_sub(x[6], x[8]);
    const float2 e = p_sub(d57, d68), o = p_add(d57, d68);
    m[3] = p_add(d13, e);
    m[4] = p_fma(-2.0f, d13, e);
    m[5] = p_add(d24, o);
    m[6] = p_fma(-2.0f, d24, o);
    m[7] = p_sub(s13, s24);
    m[8] = p_sub(s57, s68);
}

// M^-1 m for a pair of moment sets (the algebra of inverse_moments()).
__device__ __forceinline__ void inverse_moments_p(const float2* m, float2* x) {
    const float2 a0 = p_mul(1.0f / 9.0f, m[0]);
    const float2 a1 = p_mul(1.0f / 36.0f, m[1]);
    const float2 a2 = p_mul(1.0f / 36.0f, m[2]);
    const float2 a3 = p_mul(1.0f / 6.0f, m[3]);
    const float2 a4 = p_mul(1.0f / 12.0f, m[4]);
    const float2 a5 = p_mul(1.0f / 6.0f, m[5]);
    const float2 a6 = p_mul(1.0f / 12.0f, m[6]);
    const float2 a7 = p_mul(0.25f, m[7]);
    const float2 a8 = p_mul(0.25f, m[8]);
    const float2 e = p_fma(-2.0f, a2, p_sub(a0, a1));  // axis directions, isotropic part
    const float2 d = p_fma(2.0f, a1, p_add(a0, a2));   // diagonal directions, isotropic part
    const float2 jz = p_fma(-2.0f, a4, a3), jr = p_fma(-2.0f, a6, a5);
    const float2 qz = p_add(a3, a4), qr = p_add(a5, a6);
    const float2 qp = p_add(qz, qr), qm = p_sub(qz, qr);
    x[0] = p_fma(-4.0f, a1, p_fma(4.0f, a2, a0));
    const float2 ep = p_add(e, a7), em = p_sub(e, a7);
    x[1] = p_add(ep, jz);
    x[3] = p_sub(ep, jz);
    x[2] = p_add(em, jr);
    x[4] = p_sub(em, jr);
    const float2 dp = p_add(d, a8), dm = p_sub(d, a8);
    x[5] = p_add(dp, qp);
    x[7] = p_sub(dp, qp);
    x[6] = p_sub(dm, qm);
    x[8] = p_add(dm, qm);
}

// mf = M f and mg = M g: one packed transform in FP32, two scalar ones in FP64.
__device__ __forceinline__ void moments_fg(const double* f, const double* g, double* mf, double* mg) {
    moments<double>(f, mf);
    moments<double>(g, mg);
}
__device__ __forceinline__ void moments_fg(const float* f, const float* g, float* mf, float* mg) {
    float2 x[9], m[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) x[i] = make_float2(f[i], g[i]);
    moments_p(x, m);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        mf[i] = m[i].x;
        mg[i] = m[i].y;
    }
}
// f+ = M^-1 mf+ and g+ = M^-1 mg+.
__device__ __forceinline__ void inverse_moments_fg(const double* mf, const double* mg, double* f, double* g) {
    inverse_moments<double>(mf, f);
    inverse_moments<double>(mg, g);
}
__device__ __forceinline__ void inverse_moments_fg(const float* mf, const float* mg, float* f, float* g) {
    float2 m[9], x[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) m[i] = make_float2(mf[i], mg[i]);
    inverse_moments_p(m, x);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        f[i] = x[i].x;
        g[i] = x[i].y;
    }
}

// Everything before the collisions for node (k, j) of case C, from the
// shared phi window (centred on (a, b)) and the node's decoded g.
//
// RM (rate mode, lbm_internal.h): with kRatesPaper the rate pattern of the
// paper's runs (Sec. 3.1) -- S^f = diag(1, 1, 1, s, s, s, s, 1, 1) and S^g = 1
// except s1 = s7 = s8 = 1/tau_g(x) -- is known at compile time, so unit-rate
// moments go straight to their equilibrium and s_p = (s1 + s2 - s1 s2) /
// (2 s1 s2) = tau_g / 2; with kRatesPaperRaw the same choice in the raw basis
// (s_3 = 1/tau_g, s_8 = 1) gives s_p = 3 tau_g / 2 - 1.
//
// inv_r_tab: when not null, 1 / r of the node's column (a table lookup
// standing for the same correctly rounded quotient).
//
// VP (FP32 arithmetic only): the first eight scalar parameters are read from
// the 16-byte aligned FP32 block of the shared case record as two 16-byte
// loads (measured -1.1 % on the mixed FP16 step, +0.2 % in FP32 storage, so
// only the 16-bit codecs ask for it).
template <typename Real, int LD, int RM = kRatesGeneral, bool VP = false>
__device__ __forceinline__ void node_macros(const CaseDev& C, const Real* sphi, int a, int b, int j, const Real* mg,
                                            Real g0, Real p_prev, Macro<Real>& m, const Real* inv_r_tab = nullptr) {
    const CaseReal<Real>& P = case_params<Real>(C);
    static_assert(!VP || sizeof(Real) == 4, "vector parameter loads read the FP32 block");
    float4 v0{}, v1{};
    if constexpr (VP) {
        const float4* pv = reinterpret_cast<const float4*>(&C.pf);
        v0 = pv[0];
        v1 = pv[1];
    }
    m.r = (Real)j + (Real)0.5;
    m.inv_r = inv_r_tab ? *inv_r_tab : rcp_(m.r);
    m.phi = sphi[a * LD + b];
    stencil<Real, LD>(sphi, a, b, m.gz, m.gr, m.lap);
    const Real rho_l = VP ? (Real)v0.x : P.rho_l, rho_g = VP ? (Real)v0.y : P.rho_g;
    m.rho = m.phi * rho_l + ((Real)1 - m.phi) * rho_g;                    // Eq. 17
    m.nu = m.phi * (VP ? (Real)v0.z : P.nu_l) + ((Real)1 - m.phi) * (VP ? (Real)v0.w : P.nu_g);  // Eq. 35
    const Real tau_g = (Real)3 * m.nu + (Real)0.5;                         // Eq. 34
    // FP64: one reciprocal for three quotients, X = 1 / (rho (r + nu / r)
    // tau_g), gives 1 / tau_g, 1 / (r rho + nu rho / r) of Eq. 32 (r) and
    // 1 / (r rho) of Eq. 32 (z) by multiplications: two FP64 divisions (long
    // sequences on the FP64 pipe) fewer per node, -4.2 % on the FP64 step.
    // FP32 arithmetic keeps three hardware reciprocals: merging them there
    // saved 1.6 % in FP16 storage, but its rounding changes stopped the
    // bfloat16 P2 drop's oscillation and the ratio-1000 thread's breakup
    // (bfloat16's 8 bits let rounding decide whether a slowly moving
    // interface moves or stays), so the FP32 forms keep their tested numbers.
    constexpr bool kMergeRcp = sizeof(Real) == 8;
    const Real rt = m.rho * (m.r + m.nu * m.inv_r);
    // the interface normal's denominator |grad phi| + n_eps (Eq. 2)
    const Real nden = sqrt_(m.gz * m.gz + m.gr * m.gr) + (VP ? (Real)v1.y : P.n_eps);
    Real sgv, iDr, ign;
    if constexpr (kMergeRcp) {
        // one division for 1 / tau_g, 1 / (r rho + nu rho / r) and the
        // normal's 1 / nden: Y = 1 / (rho (r + nu / r) tau_g nden)
        const Real rtt = rt * tau_g;
        const Real Y = rcp_(rtt * nden);
        const Real X = Y * nden;
        sgv = X * rt;
        iDr = X * tau_g;
        ign = Y * rtt;
    } else {
        sgv = rcp_(tau_g);
        iDr = rcp_(m.r * m.rho + m.nu * m.rho * m.inv_r);
        ign = rcp_(nden);
    }
    if constexpr (RM == kRatesPaper) {
        m.sg[1] = sgv;
    } else if constexpr (RM == kRatesPaperRaw) {
        m.sg[3] = sgv;
    } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) m.sg[i] = ((C.sg_local >> i) & 1u) ? sgv : P.sg[i];
    }
    // Eq. 4 and mu~ = mu - k d_r phi / r
    const Real kap = VP ? (Real)v1.w : P.kappa;
    const Real mu = (Real)4 * (VP ? (Real)v1.z : P.beta) * m.phi * (m.phi - (Real)1) * (m.phi - (Real)0.5) - kap * m.lap;
    const Real mut = mu - kap * m.gr * m.inv_r;
    const Real Fsz = mut * m.gz, Fsr = mut * m.gr;
    const Real Gz = (m.rho - rho_l) * (VP ? (Real)v1.x : P.grav_z);
    // interface normal and lambda (Eq. 2)
    m.nzn = m.gz * ign;
    m.nrn = m.gr * ign;
    m.lam = (Real)4 * m.phi * ((Real)1 - m.phi) * P.inv_W;
    // hydrodynamic moments (M g, computed by the caller)
#pragma unroll
    for (int i = 0; i < 9; ++i) m.mg[i] = mg[i];
    const Real Jz = m.mg[3], Jr = m.mg[5], S0 = m.mg[0] - g0;
    const Real drho = rho_l - rho_g;
    const Real dzrho = drho * m.gz, drrho = drho * m.gr;
    Real sp;
    if constexpr (RM == kRatesPaper) {
        sp = (Real)0.5 * tau_g;
    } else if constexpr (RM == kRatesPaperRaw) {
        sp = (Real)1.5 * tau_g - (Real)1;  // s_3 = 1/tau_g, s_8 = 1
    } else if (C.collision == 1) {
        // raw moments: Appendix C in that basis (x_0 = k_0 - k_3 + k_8)
        sp = (Real)1.5 * rcp_(m.sg[3]) - (Real)0.5 * rcp_(m.sg[8]) - (Real)0.5;
    } else {
        const Real s1 = m.sg[1], s2 = m.sg[2];
        sp = div_(s1 + s2 - s1 * s2, (Real)2 * s1 * s2);
    }
    const Real r = m.r;
    // Eq. 32 (z); FP64: 1 / (r rho) = (1 / r) (r + nu / r) / (r rho + nu rho / r)
    if constexpr (kMergeRcp) m.uz = (Jz + (Real)0.5 * r * (Fsz + Gz)) * (m.inv_r * (iDr * (r + m.nu * m.inv_r)));
    else m.uz = div_(Jz + (Real)0.5 * r * (Fsz + Gz), r * m.rho);
    if (C.p_coupling == 1) {
        m.pstar = p_prev;
        m.ur = (Jr + (Real)0.5 * (r * Fsr + m.pstar)) * iDr;                // Eq. 32 (r)
        m.p = (Real)0.6 * (S0 * m.inv_r + (Real)0.5 * (m.uz * dzrho + m.ur * drrho) -
                           (Real)(2.0 / 3.0) * m.rho * (m.uz * m.uz + m.ur * m.ur) -
                           sp * (Real)(4.0 / 9.0) * m.rho * m.ur * m.inv_r); // Eq. 33
    } else {
        // Eq. 32 (r) and Eq. 33 together: u_r = a + b p, p = A0 + A1 u_r - A2 u_r^2
        const Real ca = (Jr + (Real)0.5 * r * Fsr) * iDr;
        const Real cb = (Real)0.5 * iDr;
        const Real A0 = (Real)0.6 * (S0 * m.inv_r + (Real)0.5 * m.uz * dzrho - (Real)(2.0 / 3.0) * m.rho * m.uz * m.uz);
        const Real A1 = (Real)0.6 * ((Real)0.5 * drrho - sp * (Real)(4.0 / 9.0) * m.rho * m.inv_r);
        const Real A2 = (Real)0.4 * m.rho;
        const Real qa = A2 * cb * cb;
        const Real qb = (Real)1 - A1 * cb + (Real)2 * A2 * ca * cb;
        const Real qc = -(A0 + A1 * ca - A2 * ca * ca);
        const Real disc = qb * qb - (Real)4 * qa * qc;
        // one division: the root's numerator and denominator are selected first
        const bool two = disc >= (Real)0;
        m.p = div_(two ? (Real)-2 * qc : -qc, two ? qb + sqrt_(disc) : qb);
        m.pstar = m.p;
        m.ur = ca + cb * m.p;
    }
    // Eq. 30
    m.Fz = r * (Fsz + Gz);
    m.Fr = r * Fsr + m.pstar - (Real)2 * m.rho * m.nu * m.ur * m.inv_r;
}

// ---------------------------------------------------------------- collisions
// Phase field (Eq. 19 in moment space with Eq. 21-23).  chi = (r phi u_z,
// r phi u_r + M phi); the time derivative of Eq. 38 uses chi^{n-1}.
template <typename Real, int RM = kRatesGeneral>
__device__ __forceinline__ void collide_f(const CaseDev& C, const Macro<Real>& m, const Real* mf, Real chi_z_prev,
                                          Real chi_r_prev, Real& chi_z, Real& chi_r, Real* mp) {
    const CaseReal<Real>& P = case_params<Real>(C);
    const Real rphi = mf[0];  // = r phi exactly (phi is sum f / r)
    chi_z = m.r * m.phi * m.uz;
    chi_r = m.r * m.phi * m.ur + P.mob * m.phi;
    const Real mR1 = (chi_z - chi_z_prev) + m.r * m.nzn * m.lam * (Real)(1.0 / 3.0);
    const Real mR2 = (chi_r - chi_r_prev) + m.r * m.nrn * m.lam * (Real)(1.0 / 3.0);
    const Real meq[9] = {rphi, (Real)-2 * rphi, rphi, chi_z, -chi_z, chi_r, -chi_r, (Real)0, (Real)0};
    const Real mR[9] = {(Real)0, (Real)0, (Real)0, mR1, -mR1, mR2, -mR2, (Real)0, (Real)0};
    if constexpr (RM != kRatesGeneral) {
        // unit rates: m0 is conserved, m1, m2, m7, m8 take their equilibria.
        // The raw-moment pattern (rate s on c_z, c_r, c_z^2 c_r, c_z c_r^2)
        // spans the same rate subspaces, so it is this very operator; its s
        // is the rate of raw moment 1.
        const Real s = RM == kRatesPaperRaw ? P.sf[1] : P.sf[3], h = (Real)1 - (Real)0.5 * s;
        mp[0] = rphi;
        mp[1] = meq[1];
        mp[2] = meq[2];
#pragma unroll
        for (int k = 3; k < 7; ++k) mp[k] = mf[k] - s * (mf[k] - meq[k]) + h * mR[k];
        mp[7] = (Real)0;
        mp[8] = (Real)0;
    } else if (C.collision == 1) {
        raw_relax<Real>(mf, meq, mR, P.sf, mp);
    } else {
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const Real s = P.sf[k];
            mp[k] = mf[k] - s * (mf[k] - meq[k]) + ((Real)1 - (Real)0.5 * s) * mR[k];
        }
    }
}

// Hydrodynamics (Eq. 24 in moment space with Eq. 36-37).
template <typename Real, int RM = kRatesGeneral>
__device__ __forceinline__ void collide_g(const CaseDev& C, const Macro<Real>& m, Real* mp) {
    const CaseReal<Real>& P = case_params<Real>(C);
    const Real r = m.r, rho = m.rho, uz = m.uz, ur = m.ur, p = m.p;
    const Real u2 = uz * uz + ur * ur;
    const Real drho = P.rho_l - P.rho_g;
    const Real dz_rr = r * drho * m.gz;          // d_z (r rho)
    const Real dr_rr = rho + r * drho * m.gr;    // d_r (r rho)
    const Real udr = uz * dz_rr + ur * dr_rr;
    const Real meq[9] = {(Real)0,
                         r * (Real)3 * ((Real)2 * p + rho * u2),
                         -r * (Real)3 * ((Real)3 * p + rho * u2),
                         r * rho * uz, -r * rho * uz,
                         r * rho * ur, -r * rho * ur,
                         r * rho * (uz * uz - ur * ur),
                         r * rho * ur * uz};
    const Real MT[9] = {udr - rho * ur,  // = r u . grad rho
                        (Real)2 * rho * ur,
                        -udr - rho * ur,
                        m.Fz, -m.Fz, m.Fr, -m.Fr,
                        (Real)(2.0 / 3.0) * (uz * dz_rr - ur * dr_rr),
                        (Real)(1.0 / 3.0) * (uz * dr_rr + ur * dz_rr)};
    if constexpr (RM == kRatesPaper) {
        const Real s = m.sg[1], h = (Real)1 - (Real)0.5 * s;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            if (k == 1 || k == 7 || k == 8) mp[k] = m.mg[k] - s * (m.mg[k] - meq[k]) + h * MT[k];
            else mp[k] = meq[k] + (Real)0.5 * MT[k];
        }
    } else if constexpr (RM == kRatesPaperRaw) {
        // raw moments: the three second moments at 1/tau_g, the rest at 1
        const Real s = m.sg[3];
        const Real rates[9] = {(Real)1, (Real)1, (Real)1, s, s, s, (Real)1, (Real)1, (Real)1};
        raw_relax<Real>(m.mg, meq, MT, rates, mp);
    } else if (C.collision == 1) {
        raw_relax<Real>(m.mg, meq, MT, m.sg, mp);
    } else {
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const Real s = m.sg[k];
            mp[k] = m.mg[k] - s * (m.mg[k] - meq[k]) + ((Real)1 - (Real)0.5 * s) * MT[k];
        }
    }
}

// ---------------------------------------------------------------- streaming
// Push f+_i(k, j) along c_i (Eq. 20).  A link that leaves through a wall (the
// z-walls when not periodic, the wall r = nr, and any corner) is bounced back
// to its own node as direction opp(i); a link that leaves through the axis
// alone enters (k + c_z, 0) as the r-mirrored direction.
struct Dest {
    int k, j, dir;
};
template <int I>
__device__ __forceinline__ Dest destination(int k, int j, int nr, int nz, int zper) {
    int kt = k + cz_of(I);
    const int jt = j + cr_of(I);
    bool zout = false;
    if (cz_of(I) != 0) {
        if (zper) {
            kt = kt < 0 ? kt + nz : (kt >= nz ? kt - nz : kt);
        } else {
            zout = (kt < 0) || (kt >= nz);
        }
    }
    const bool rwall = (cr_of(I) > 0) && (jt >= nr);
    if (zout || rwall) return Dest{k, j, opp_of(I)};
    if (cr_of(I) < 0 && jt < 0) return Dest{kt, 0, rmir_of(I)};
    return Dest{kt, jt, I};
}

// ---------------------------------------------------------------- TMA / mbarrier
// Bulk tensor copies global -> shared completed on an mbarrier (PTX ISA,
// sm_90 and later).  One elected thread issues them; every thread waits on the
// barrier's phase with a bounded number of tries.
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// Wait for phase `phase` of the barrier; gives up after `limit` tries and
// reports it through *status (the host turns it into LBM_ERR_TIMEOUT).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t phase, int* status, int limit) {
    for (int i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, phase)) return true;
    atomicExch(status, 1);
    return false;
}

__device__ __forceinline__ void tensormap_acquire(const CUtensorMap* map) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"((uint64_t)map) : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_addr(dst)),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_addr(dst)),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(smem_addr(dst)),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
        : "memory");
}

// Prefetch a tensor box into L2 (no shared-memory destination, no completion).
__device__ __forceinline__ void tma_prefetch_4d(const CUtensorMap* map, int c0, int c1, int c2, int c3) {
    asm volatile("cp.async.bulk.prefetch.tensor.4d.L2.global.tile [%0, {%1, %2, %3, %4}];" ::"l"((uint64_t)map),
                 "r"(c0), "r"(c1), "r"(c2), "r"(c3)
                 : "memory");
}

// Plain bulk copy global -> shared (no tensor map): both addresses 16-byte
// aligned, `bytes` a multiple of 16; completes on `bar`.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"((uint64_t)src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

}  // namespace axilbm
