// lbm_kernels.cuh -- kernel templates of the step, the field recovery, the
// initial condition and the state transfer.  Each precision's .cu file
// includes this header and instantiates the launchers for its codec.
#pragma once

#include <cuda_runtime.h>

#include "lbm_device.cuh"
#include "lbm_internal.h"
#include "lbm_lane.cuh"

namespace axilbm {

constexpr int kTR = 32;  // tile width along r = one warp
// L2 prefetch distance of the step in quarters of a resident wave of CTAs
// (SMs x CTAs per SM).  Measured on the 512-case batch: anything from 3/4 to
// 3/2 of a wave gives the same time, half a wave or two waves less.  With
// FP16's grid codec (ms per step, one node per thread): 2 quarters 0.751,
// 4 0.723, 8 0.721, 16 0.755; FP32 (two nodes per thread) 0.731, 0.733,
// 0.955, 0.972.  AXILBM_PREFETCH_QUARTERS overrides it for tuning builds.
#ifndef AXILBM_PREFETCH_QUARTERS
#define AXILBM_PREFETCH_QUARTERS 4
#endif
constexpr int kPrefetchQuarters = AXILBM_PREFETCH_QUARTERS;

// Column constants of the 16-bit grid codecs (GridCol) for the window
// columns b = 0 .. kTR + 3 of a tile (column ghost_r(j0 - 2 + b)), built
// once per CTA in shared memory as three arrays, so a warp's lookups of
// consecutive columns are conflict-free 16-byte loads.
struct GridTab {
    float4* A;  // invS_a, G_a, cS_a, S_a
    float4* D;  // invS_d, G_d, cS_d, S_d
    uint4* H;   // S16, S16g, S16g0, -
    __device__ __forceinline__ GridCol col(int b) const {
        const float4 a = A[b], d = D[b];
        const uint4 h = H[b];
        return GridCol{a.x, a.y, a.z, a.w, d.x, d.y, d.z, d.w, h.x, h.y, h.z, h.w};
    }
    __device__ __forceinline__ void put(int b, const GridCol& g) const {
        A[b] = make_float4(g.invS_a, g.G_a, g.cS_a, g.S_a);
        D[b] = make_float4(g.invS_d, g.G_d, g.cS_d, g.S_d);
        H[b] = make_uint4(g.S16, g.S16g, g.S16g0, g.pad);
    }
};
template <class Codec>
__device__ __forceinline__ void grid_tab_fill(const GridTab& T, int q, int j0, int nr) {
    if (q < kTR + 4) T.put(q, grid_col<Codec>(ghost_r(j0 - 2 + q, nr)));
}

// Where node_update takes the column constants of the three columns a node's
// populations land in (s = 0: the column j - 1, or j on the axis; s = 1: j;
// s = 2: j + 1, or j at the wall r = nr): none (FP64, FP32), a GridTab, or
// computed from the column index.
struct NoCols {
    __device__ __forceinline__ GridCol get(int) const { return GridCol{}; }
};
struct TabCols {
    GridTab T;
    int bm, bo, bp;
    __device__ __forceinline__ GridCol get(int s) const { return T.col(s == 0 ? bm : (s == 1 ? bo : bp)); }
};
template <class Codec>
struct CalcCols {
    int jm, jo, jp;
    __device__ __forceinline__ GridCol get(int s) const { return grid_col<Codec>(s == 0 ? jm : (s == 1 ? jo : jp)); }
};

// phi of node (k, j) at storage index loc, with everything taken from j
template <class Codec>
__device__ __forceinline__ typename Codec::Real node_phi_at(const CaseView<Codec>& V, int loc, int j) {
    using Real = typename Codec::Real;
    const Real r = (Real)j + (Real)0.5;
    float Sa = 0.0f;
    if constexpr (Codec::kGrid) Sa = grid_sa<Codec>(j);
    return node_phi<Codec>(V.in_node(loc), rcp_(r), Sa);
}

// phi at window position (a, b) of tile t through the ghost rules.
template <class Codec>
__device__ __forceinline__ typename Codec::Real window_phi(const CaseDev& C, const CaseView<Codec>& V,
                                                            const TileDev& t, int a, int b) {
    const int k = ghost_z(t.k0 - 2 + a, C.nz, C.zper);
    const int j = ghost_r(t.j0 - 2 + b, C.nr);
    return node_phi_at<Codec>(V, k * C.pitch + j, j);
}

// The ring of a tile's phi window: the two rows above and below the tile and
// the two columns left and right of it, 4 * 32 + 4 * (TZ + 4) cells.  Cell q
// maps to window position (a, b): first the 32 middle cells of each of the
// four halo rows (one warp per row, lane = column, so a warp's loads are one
// coalesced run and its ghost row is warp-uniform), then the two edge cells on
// each side of every window row.
template <int TZ>
__device__ __forceinline__ void ring_cell(int q, int& a, int& b) {
    if (q < 4 * kTR) {
        const int w = q / kTR;
        a = w < 2 ? w : TZ + w;
        b = 2 + q % kTR;
    } else {
        const int q2 = q - 4 * kTR;
        a = q2 >> 2;
        const int c = q2 & 3;
        b = c < 2 ? c : kTR + c;
    }
}

// Minimum resident CTAs per SM requested from the register allocator.  The
// FP32-arithmetic kernels with a compile-time rate pattern take 5 CTAs of 8
// rows (40 warps per SM, 48 registers a thread, a few bytes of spill): against
// 4 CTAs (64 registers, no spill) that measured -3.4 % in FP32, -2.2 % in
// FP16 and -5.1 % in BF16 storage with the paper's collision, with the same
// results.  The raw-moment collision in bfloat16 storage spills more at 48
// registers and keeps 4 CTAs (0.772 against 0.817 ms); with FP16's grid
// codec it took 5 (0.778 against 0.802 ms) until the loads-first window
// phase (see below).  General rates: 4 CTAs
// of 8 rows (64 registers, a few bytes of spill): on the 512-case batch with
// every rate equal, -10.6 % in FP32 and -8.6 % in FP16 storage against 3 CTAs
// at 80 registers.  AXILBM_GENERAL_CTAS overrides the count when building for
// tuning.
#ifndef AXILBM_GENERAL_CTAS
#define AXILBM_GENERAL_CTAS 4
#endif
// With the loads-first window phase the one-node FP16 kernels spill at 48
// registers: 4 CTAs measured 0.763 against 0.792 ms (paper's collision) and
// 0.798 against 0.874 ms (raw moments), while bfloat16 keeps 5 (0.734 against
// 0.776 ms).  AXILBM_STEP16_CTAS (bfloat16) and AXILBM_GRID16_CTAS (FP16's
// grid codec, both collisions) override the counts for tuning builds.
#ifndef AXILBM_STEP16_CTAS
#define AXILBM_STEP16_CTAS 5
#endif
#ifndef AXILBM_GRID16_CTAS
#define AXILBM_GRID16_CTAS 4
#endif
template <class Codec, int BZ, int RM>
constexpr int step_min_blocks() {
    constexpr int bz8 = Codec::kGrid ? AXILBM_GRID16_CTAS
                        : (RM == kRatesPaperRaw && sizeof(typename Codec::PT) == 2)
                            ? 4
                            : (sizeof(typename Codec::PT) == 2 ? AXILBM_STEP16_CTAS : 5);
    return sizeof(typename Codec::Real) == 8 ? 1
           : RM != kRatesGeneral ? (BZ >= 16 ? 2 : (BZ >= 8 ? bz8 : 8))
                : (BZ >= 16 ? 1 : (BZ >= 8 ? AXILBM_GENERAL_CTAS : 2 * AXILBM_GENERAL_CTAS));
}

// Store one post-collision population pair (f_i, g_i) in the slot `dst` of
// its destination (one vector store), with the destination radius
// normalisation wr / iw.  Returns f_i as the reader will decode it (for the
// mass ledger).
template <class Codec>
__device__ __forceinline__ typename Codec::Real store_pair(typename Codec::PT2* dst, typename Codec::Real wr,
                                                           typename Codec::Real iw, typename Codec::Real fpi,
                                                           typename Codec::Real gpi) {
    const typename Codec::PT2 e = Codec::enc_pair(fpi, gpi, wr, iw);
    if constexpr (Codec::kStreamStores) __stcs(dst, e);
    else *dst = e;
    return Codec::dec_f(e.x, wr);
}
// The same for the 16-bit grid codecs, with the destination column's constants.
template <class Codec>
__device__ __forceinline__ float store_pair_grid(typename Codec::PT2* dst, const GridCol& g, bool D, float fpi,
                                                 float gpi) {
    const typename Codec::PT2 e = Codec::enc_pair(fpi, gpi, g, D);
    if constexpr (Codec::kStreamStores) __stcs(dst, e);
    else *dst = e;
    return Codec::dec_f(e.x, g, D);
}

// Direction I's store of the branch-free push in either storage form: the
// radii rdst / rinv (s = cr_of(I) + 1) or the column constants cols.get(s).
template <class Codec, int I, class Cols>
__device__ __forceinline__ typename Codec::Real store_dir(typename Codec::PT2* dst, const Cols& cols,
                                                          const typename Codec::Real* rdst,
                                                          const typename Codec::Real* rinv, typename Codec::Real f,
                                                          typename Codec::Real g) {
    using Real = typename Codec::Real;
    if constexpr (Codec::kGrid) {
        return store_pair_grid<Codec>(dst, cols.get(cr_of(I) + 1), I > 4, f, g);
    } else {
        return store_pair<Codec>(dst, (Real)w_of(I) * rdst[cr_of(I) + 1], (Real)(1.0 / w_of(I)) * rinv[cr_of(I) + 1],
                                 f, g);
    }
}

// Byte offset of direction d's pair slot inside a node group's block.
template <class Codec>
__device__ __forceinline__ constexpr int pair_slot_of(int d) {
    return Block<Codec>::off_pairs + (d - 1) * Block<Codec>::pair_slot;
}

// Where the post-collision pair I of a node lands, as a byte offset from the
// node's own pair pointer, for a node outside the z-wall rows: along c_i to
// its neighbour (rz and the lane steps: the z row step, already wrapped for
// periodic z, and the step to the next or previous lane, which crosses into
// the adjacent block at lanes 31 and 0); through the wall r = nr back to the
// node itself as direction opp(I); through the axis into row 0 of the
// destination z row as the r-mirrored direction (Sec. 2.3).
template <class Codec, int I>
__device__ __forceinline__ int push_offset(bool axis, bool wall, int rowp, int rowm, int step_r, int step_l) {
    static_assert(I != 0, "the rest populations stay at their node");
    constexpr int cz = cz_of(I), cr = cr_of(I);
    const int rz = cz > 0 ? rowp : (cz < 0 ? rowm : 0);
    if constexpr (cr > 0) return wall ? pair_slot_of<Codec>(opp_of(I)) : rz + step_r + pair_slot_of<Codec>(I);
    else if constexpr (cr < 0) return rz + (axis ? pair_slot_of<Codec>(rmir_of(I)) : step_l + pair_slot_of<Codec>(I));
    else return rz + pair_slot_of<Codec>(I);
}

// What the collisions take from a node's own populations: the moments M f and
// M g, g_0, and the FP32 mass ledger's incoming total.  The FP32 ledger is two
// double-float lanes (f_0 with f_1..4, and f_5..8) advanced together, exact;
// in 16-bit storage M f's first moment is the ledger's incoming total itself
// (exact sums on the grid).  Decoded populations die here, which keeps the
// register pressure of the collisions down.  fdec: f_0..8 already decoded by
// the caller (it summed them for phi), else decoded here.  go: the node's own
// column constants (16-bit storage).
template <typename Real>
struct PreCollision {
    Real mf[9], mg[9];
    Real g0;
    FF2 ledger;
};
template <class Codec>
__device__ __forceinline__ void node_pre(const typename Codec::F0T& f0raw, const typename Codec::PT* fraw,
                                         const typename Codec::PT* graw, typename Codec::Real r,
                                         PreCollision<typename Codec::Real>& P, const typename Codec::Real* fdec,
                                         const GridCol& go) {
    using Real = typename Codec::Real;
    Real f[9], g[9];
    if (fdec != nullptr) {
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = fdec[i];
    } else {
        f[0] = (Real)f0_value(f0raw);
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            if constexpr (Codec::kGrid) f[i] = Codec::dec_f(fraw[i - 1], go, i > 4);
            else f[i] = Codec::dec_f(fraw[i - 1], (Real)w_of(i) * r);
        }
    }
    if constexpr (Codec::kGrid) {
        g[0] = Codec::dec_g0(graw[0], go);
#pragma unroll
        for (int i = 1; i < 9; ++i) g[i] = Codec::dec_g(graw[i], go, i > 4);
    } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = Codec::dec_g(graw[i], (Real)w_of(i) * r);
    }
    moments_fg(f, g, P.mf, P.mg);
    P.g0 = g[0];
    P.ledger = FF2{};
    if constexpr (Codec::kLedger) {
        P.ledger = FF2{make_float2(((const float2&)f0raw).x, 0.0f), make_float2(((const float2&)f0raw).y, 0.0f)};
#pragma unroll
        for (int i = 1; i < 5; ++i) ff2_add(P.ledger, make_float2((float)f[i], (float)f[i + 4]));
    }
}

// Steps a4-a10 for one node whose raw stored values have been fetched: decode,
// macroscopic recovery, both collisions, and the push with the boundary rules.
// invr: when not null, 1 / r of window column b - 1, b, b + 1 at invr[b - 1 ..
// b + 1] (the same quotients the node would compute itself).  fdec: see
// node_pre.  cols: the column constants of the 16-bit grid codecs (NoCols
// otherwise).
template <class Codec, int RM, int LD, class Cols>
__device__ __forceinline__ void node_update_pre(const CaseDev& C, const CaseView<Codec>& V,
                                                const typename Codec::Real* sphi, int a, int b, int k, int j, int loc,
                                                const PreCollision<typename Codec::Real>& pre,
                                                typename Codec::Real chz_prev, typename Codec::Real chr_prev,
                                                typename Codec::Real p_prev, const typename Codec::Real* invr,
                                                const Cols& cols) {
    using Real = typename Codec::Real;
    const Real r = (Real)j + (Real)0.5;
    const Real* mf = pre.mf;
    Macro<Real> m;
    node_macros<Real, LD, RM, sizeof(typename Codec::PT) == 2>(C, sphi, a, b, j, pre.mg, pre.g0, p_prev, m,
                                                               invr ? invr + b : nullptr);
    FF2 ledger = pre.ledger;
    Real mpf[9], chz, chr;
    collide_f<Real, RM>(C, m, mf, chz_prev, chr_prev, chz, chr, mpf);
    const Node<Codec> own = V.out_node(loc);
    own.chz() = chz;
    own.chr() = chr;
    if (C.p_coupling == 1) own.p() = m.p;
    Real mpg[9];
    collide_g<Real, RM>(C, m, mpg);
    Real fp[9], gp[9];
    inverse_moments_fg(mpf, mpg, fp, gp);
    // 5. streaming (Eq. 20).  Rows j-1, j, j+1 are the only destinations, so
    //    three radii (three columns' constants in 16-bit storage) serve every
    //    normalisation.  On the axis every link with c_r < 0 ends in the
    //    node's own row (mirror) or at the node itself (bounce-back), and on
    //    the wall r = nr every link with c_r > 0 returns to the node, so there
    //    the row's own radius takes the place of the missing neighbour row.
    const bool axis = (j == 0), wall = (j + 1 == C.nr), zlo = (k == 0), zhi = (k + 1 == C.nz);
    const Real rinv[3] = {axis ? m.inv_r : (invr ? invr[b - 1] : rcp_(r - (Real)1)), m.inv_r,
                          wall ? m.inv_r : (invr ? invr[b + 1] : rcp_(r + (Real)1))};
    const Real rdst[3] = {axis ? r : r - (Real)1, r, wall ? r : r + (Real)1};
    using PT2 = typename Codec::PT2;
    constexpr int kB = Block<Codec>::bytes, kPS = (int)sizeof(PT2);
    const int lane = loc & 31;
    unsigned char* const q0 = V.out_pt(loc).q;  // the node's own pair pointer
    const int row = (C.pitch >> 5) * kB;         // one z row of blocks
    const int step_r = lane == 31 ? kB - 31 * kPS : kPS;
    const int step_l = lane == 0 ? -(kB - 31 * kPS) : -kPS;
    // 16-bit grid codecs: the ledger is M f's first moment minus the stored
    // outgoing f_1..8 (exact), summed by direction pairs (i, i + 4)
    float2 out_acc;
    if ((zlo || zhi) && !C.zper) {
        // A z-wall row (the whole warp: a warp is one row of a tile): every
        // link by the rules of destination().
        Real fs[9];
#define AXILBM_PUSH(I)                                                                                 \
    {                                                                                                  \
        const Dest d = destination<I>(k, j, C.nr, C.nz, C.zper);                                       \
        const int s = d.j - j + 1;                                                                     \
        PT2* const dst = &V.out_pt(d.k * C.pitch + d.j).pair(d.dir);                                   \
        if constexpr (Codec::kGrid) {                                                                  \
            fs[I] = store_pair_grid<Codec>(dst, cols.get(s), (I) > 4, fp[I], gp[I]);                    \
        } else {                                                                                       \
            const Real rd = s == 0 ? rdst[0] : (s == 1 ? rdst[1] : rdst[2]);                           \
            const Real ri = s == 0 ? rinv[0] : (s == 1 ? rinv[1] : rinv[2]);                           \
            fs[I] = store_pair<Codec>(dst, (Real)w_of(I) * rd, (Real)(1.0 / w_of(I)) * ri, fp[I], gp[I]); \
        }                                                                                              \
    }
        AXILBM_PUSH(1)
        AXILBM_PUSH(2)
        AXILBM_PUSH(3)
        AXILBM_PUSH(4)
        AXILBM_PUSH(5)
        AXILBM_PUSH(6)
        AXILBM_PUSH(7)
        AXILBM_PUSH(8)
#undef AXILBM_PUSH
#pragma unroll
        for (int i = 1; i < 5; ++i) {
            if constexpr (Codec::kLedger) ff2_sub(ledger, make_float2((float)fs[i], (float)fs[i + 4]));
            if constexpr (Codec::kExactLedger)
                out_acc = i == 1 ? make_float2(fs[i], fs[i + 4]) : p_add(out_acc, make_float2(fs[i], fs[i + 4]));
        }
    } else {
        // Every other node, branch-free: the axis and wall lanes differ from
        // their warp only in the offsets of push_offset(), and a z row that
        // wraps (periodic z) only in its row steps.  The ledger takes each
        // pair of directions (i, i + 4) as soon as both are stored.
        const int rowp = zhi ? -(C.nz - 1) * row : row;
        const int rowm = zlo ? (C.nz - 1) * row : -row;
#define AXILBM_DST(I) reinterpret_cast<PT2*>(q0 + push_offset<Codec, I>(axis, wall, rowp, rowm, step_r, step_l))
#define AXILBM_STORE(I) store_dir<Codec, I>(AXILBM_DST(I), cols, rdst, rinv, fp[I], gp[I])
#define AXILBM_STORE_TWO(I)                                                                              \
    {                                                                                                    \
        const Real fa = AXILBM_STORE(I), fb = AXILBM_STORE(I + 4);                                       \
        if constexpr (Codec::kLedger) ff2_sub(ledger, make_float2((float)fa, (float)fb));                \
        if constexpr (Codec::kExactLedger) out_acc = (I) == 1 ? make_float2(fa, fb) : p_add(out_acc, make_float2(fa, fb)); \
    }
        AXILBM_STORE_TWO(1)
        AXILBM_STORE_TWO(2)
        AXILBM_STORE_TWO(3)
        AXILBM_STORE_TWO(4)
#undef AXILBM_STORE_TWO
#undef AXILBM_STORE
#undef AXILBM_DST
    }
    // the rest direction: g_0 stays at the node
    {
        typename Codec::PT e0;
        if constexpr (Codec::kGrid) e0 = Codec::enc_g0(gp[0], cols.get(1));
        else e0 = Codec::enc_g(gp[0], (Real)w_of(0) * r, (Real)(1.0 / w_of(0)) * m.inv_r);
        if constexpr (Codec::kStreamStores) __stcs(&own.g(0), e0);
        else own.g(0) = e0;
    }
    // f_0: the collision's value (FP64), or the mass ledger: incoming total
    // minus the outgoing f_1..8 as they will be read back
    if constexpr (Codec::kExactLedger) {
        own.f0() = __fsub_rn(mf[0], __fadd_rn(out_acc.x, out_acc.y));
    } else if constexpr (Codec::kLedger) {
        const FF l = ff2_merge(ledger);
        own.f0() = make_float2(l.hi, l.lo);
    } else {
        own.f0() = fp[0];
    }
}

// The same from the node's raw stored values (node_pre first).
template <class Codec, int RM, int LD, class Cols>
__device__ __forceinline__ void node_update(const CaseDev& C, const CaseView<Codec>& V, const typename Codec::Real* sphi,
                                            int a, int b, int k, int j, int loc,
                                            const typename Codec::F0T& f0raw, const typename Codec::PT* fraw,
                                            const typename Codec::PT* graw, typename Codec::Real chz_prev,
                                            typename Codec::Real chr_prev, typename Codec::Real p_prev,
                                            const typename Codec::Real* invr, const typename Codec::Real* fdec,
                                            const Cols& cols) {
    PreCollision<typename Codec::Real> pre;
    node_pre<Codec>(f0raw, fraw, graw, (typename Codec::Real)j + (typename Codec::Real)0.5, pre, fdec, cols.get(1));
    node_update_pre<Codec, RM, LD>(C, V, sphi, a, b, k, j, loc, pre, chz_prev, chr_prev, p_prev, invr, cols);
}

// The stores of one FP16 node after its collisions (step a10 with the grid
// codec; fp, gp the post-collision populations): chi^n and p^n, g_0, the
// eight pushed (f_i, g_i) pairs with the boundary rules of node_update, and
// f_0 = M f's first moment (mf0, the incoming total) minus the stored
// outgoing f_1..8, exact on the grid.
template <class Codec, class Cols>
__device__ __forceinline__ void node_post_grid(const CaseDev& C, const CaseView<Codec>& V, int k, int j, int loc,
                                               const float* fp, const float* gp, float chz, float chr, float p,
                                               float mf0, const Cols& cols) {
    const Node<Codec> own = V.out_node(loc);
    own.chz() = chz;
    own.chr() = chr;
    if (C.p_coupling == 1) own.p() = p;
    const bool axis = (j == 0), wall = (j + 1 == C.nr), zlo = (k == 0), zhi = (k + 1 == C.nz);
    using PT2 = typename Codec::PT2;
    constexpr int kB = Block<Codec>::bytes, kPS = (int)sizeof(PT2);
    const int lane = loc & 31;
    unsigned char* const q0 = V.out_pt(loc).q;  // the node's own pair pointer
    const int row = (C.pitch >> 5) * kB;         // one z row of blocks
    const int step_r = lane == 31 ? kB - 31 * kPS : kPS;
    const int step_l = lane == 0 ? -(kB - 31 * kPS) : -kPS;
    float2 out_acc;  // the stored outgoing f of direction pairs (i, i + 4)
    if ((zlo || zhi) && !C.zper) {
        float fs[9];
#define AXILBM_PUSH(I)                                                                        \
    {                                                                                         \
        const Dest d = destination<I>(k, j, C.nr, C.nz, C.zper);                              \
        fs[I] = store_pair_grid<Codec>(&V.out_pt(d.k * C.pitch + d.j).pair(d.dir), cols.get(d.j - j + 1), \
                                       (I) > 4, fp[I], gp[I]);                                \
    }
        AXILBM_PUSH(1)
        AXILBM_PUSH(2)
        AXILBM_PUSH(3)
        AXILBM_PUSH(4)
        AXILBM_PUSH(5)
        AXILBM_PUSH(6)
        AXILBM_PUSH(7)
        AXILBM_PUSH(8)
#undef AXILBM_PUSH
        out_acc = make_float2(fs[1], fs[5]);
#pragma unroll
        for (int i = 2; i < 5; ++i) out_acc = p_add(out_acc, make_float2(fs[i], fs[i + 4]));
    } else {
        const int rowp = zhi ? -(C.nz - 1) * row : row;
        const int rowm = zlo ? (C.nz - 1) * row : -row;
#define AXILBM_STORE(I)                                                                                    \
    store_pair_grid<Codec>(reinterpret_cast<PT2*>(q0 + push_offset<Codec, I>(axis, wall, rowp, rowm, step_r, step_l)), \
                           cols.get(cr_of(I) + 1), (I) > 4, fp[I], gp[I])
#define AXILBM_STORE_TWO(I)                                                                          \
    {                                                                                                \
        const float fa = AXILBM_STORE(I), fb = AXILBM_STORE(I + 4);                                  \
        out_acc = (I) == 1 ? make_float2(fa, fb) : p_add(out_acc, make_float2(fa, fb));              \
    }
        AXILBM_STORE_TWO(1)
        AXILBM_STORE_TWO(2)
        AXILBM_STORE_TWO(3)
        AXILBM_STORE_TWO(4)
#undef AXILBM_STORE_TWO
#undef AXILBM_STORE
    }
    {
        const typename Codec::PT e0 = Codec::enc_g0(gp[0], cols.get(1));
        if constexpr (Codec::kStreamStores) __stcs(&own.g(0), e0);
        else own.g(0) = e0;
    }
    own.f0() = __fsub_rn(mf0, __fadd_rn(out_acc.x, out_acc.y));
}

// node_update for the FP16 grid codec: the same steps, with the macroscopic
// step and both collisions in the explicit operations of lbm_lane.cuh (one
// lane), so the packed two-node kernel computes the same numbers.
template <class Codec, int RM, int LD, class Cols>
__device__ __forceinline__ void node_update_grid(const CaseDev& C, const CaseView<Codec>& V, const float* sphi, int a,
                                                 int b, int k, int j, int loc, const typename Codec::F0T& f0raw,
                                                 const typename Codec::PT* fraw, const typename Codec::PT* graw,
                                                 float chz_prev, float chr_prev, float p_prev, const float* fdec,
                                                 const Cols& cols) {
    static_assert(Codec::kGrid, "the grid codec's update");
    PreCollision<float> pre;
    node_pre<Codec>(f0raw, fraw, graw, (float)j + 0.5f, pre, fdec, cols.get(1));
    lane::Macro<float> m;
    lane::node_macros<float, LD, RM, true>(C, sphi, a, b, j, pre.mg, pre.g0, p_prev, m);
    float mpf[9], mpg[9], chz, chr;
    lane::collide_f<float, RM>(C, m, pre.mf, chz_prev, chr_prev, chz, chr, mpf);
    lane::collide_g<float, RM>(C, m, mpg);
    float fp[9], gp[9];
    inverse_moments_fg(mpf, mpg, fp, gp);
    node_post_grid<Codec>(C, V, k, j, loc, fp, gp, chz, chr, m.p, pre.mf[0], cols);
}

// One time step for every node of every tile in `tiles`: one CTA per tile of
// BZ rows (z) x 32 columns (r), one node per thread.  Each thread first issues
// the loads of its own node; the node's phi goes to the shared window straight
// from those registers and only the two-node ring around the tile is
// recomputed from neighbours' populations.
template <class Codec, int BZ, int RM>
__global__ void __launch_bounds__(kTR * BZ, (step_min_blocks<Codec, BZ, RM>()))
step_kernel(const CaseDev* __restrict__ cases, const TileDev* __restrict__ tiles, StateDev<Codec> S,
            const CUtensorMap* __restrict__ maps, int map_set, int parity, int ntiles, int ahead) {
    using Real = typename Codec::Real;
    using PT = typename Codec::PT;
    using F0T = typename Codec::F0T;
    constexpr int TZ = BZ;
    constexpr int LD = kTR + 4;
    constexpr int NRING = 4 * kTR + 4 * (TZ + 4);
    static_assert(NRING == (TZ + 4) * LD - TZ * kTR, "the ring is the window without the tile");
    __shared__ Real sphi[(TZ + 4) * LD];
    // The case's parameters go to shared memory: read from there, the
    // collision's many per-case constants need no global loads.
    __shared__ __align__(16) CaseDev sC;
    static_assert(sizeof(CaseDev) % 4 == 0 && sizeof(CaseDev) / 4 <= kTR * BZ, "one word per thread");
    // FP64: 1 / r of the window's columns j0 - 2 .. j0 + 33, one division per
    // column instead of four per node (a division is a long sequence on the
    // FP64 pipe); the same correctly rounded quotients the nodes would form
    constexpr bool kInvrTable = sizeof(Real) == 8;
    __shared__ Real s_invr[kInvrTable ? LD : 1];
    // 16-bit storage: the column constants of the window's columns
    constexpr bool kG = Codec::kGrid;
    __shared__ float4 sgA[kG ? LD : 1], sgD[kG ? LD : 1];
    __shared__ uint4 sgH[kG ? LD : 1];
    const GridTab T{sgA, sgD, sgH};
    const TileGeo g = reinterpret_cast<const TileGeo*>(tiles + ntiles)[blockIdx.x];
    const int q = threadIdx.y * kTR + threadIdx.x;
    constexpr int kCW = (int)(sizeof(CaseDev) / 4);                // words of the case record
    constexpr int kRC = (NRING + kTR * BZ - 1) / (kTR * BZ);        // ring cells per thread
    constexpr int kB = Block<Codec>::bytes;
    // 1. every global load of the window phase leaves before any of them is
    //    used, addressed from the tile's TileGeo record alone: this thread's
    //    word of the case record, the node's own values (out of the domain:
    //    its ghost node's f), and the f of this thread's ring cells
    int32_t cw = 0;
    if (q < kCW) cw = reinterpret_cast<const int32_t*>(cases + g.c)[q];
    // L2 prefetch of the blocks of the tile one resident wave ahead (a CTA
    // that will start about when this one ends): one tensor prefetch, issued
    // by one thread; the tensor maps are absent when they could not be made
    if (maps != nullptr && q == 0 && (int)blockIdx.x + ahead < ntiles) {
        const TileDev tp = tiles[blockIdx.x + ahead];
        const CUtensorMap* M = maps + ((size_t)tp.c * 2 + map_set) * kMapsPerCase + 2 + parity;
        tensormap_acquire(M);
        tma_prefetch_4d(M, 0, 0, tp.j0 >> 5, tp.k0);
    }
    unsigned char* const base = const_cast<unsigned char*>(S.in) + (int64_t)g.blk0 * kB;  // the case's first block
    auto node_at = [&](int kk, int jj) { return Node<Codec>{base + (int64_t)(kk * g.rowblk + (jj >> 5)) * kB, jj & 31}; };
    const int j = g.j0 + threadIdx.x;
    const int k = g.k0 + threadIdx.y;
    const bool inside = (j < g.nr) && (k < g.nz);
    F0T f0raw{};
    PT fraw[8], graw[9];
    Real chz_prev = (Real)0, chr_prev = (Real)0, p_prev = (Real)0;
    if (inside) {
        const Node<Codec> n = node_at(k, j);
        f0raw = n.f0();
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            const typename Codec::PT2 pr = n.pair(i);  // (f_i, g_i) in one load
            fraw[i - 1] = pr.x;
            graw[i] = pr.y;
        }
        graw[0] = n.g(0);
        chz_prev = n.chz();
        chr_prev = n.chr();
    } else {
        load_phi_raw<Codec>(node_at(ghost_z(k, g.nz, g.zper), ghost_r(j, g.nr)), f0raw, fraw);
    }
    // 2. the window: this thread's ring cells (two rows above and below, two
    //    columns left and right of the tile), then the node's own phi (Eq.
    //    16), as soon as their loads land; 16-bit grid storage takes S_a of a
    //    column from grid_sa, the value the column table holds
    auto sa_of = [&](int jj) -> float {
        if constexpr (kG) return grid_sa<Codec>(jj);
        else return 0.0f;
    };
#pragma unroll
    for (int c = 0; c < kRC; ++c) {
        if (q + c * kTR * BZ < NRING) {
            int ra, rb;
            ring_cell<TZ>(q + c * kTR * BZ, ra, rb);
            const int rj = ghost_r(g.j0 - 2 + rb, g.nr);
            F0T rf0;
            PT rf[8];
            load_phi_raw<Codec>(node_at(ghost_z(g.k0 - 2 + ra, g.nz, g.zper), rj), rf0, rf);
            sphi[ra * LD + rb] = phi_of<Codec>(rf0, rf, rcp_((Real)rj + (Real)0.5), sa_of(rj));
        }
    }
    const Real r = (Real)j + (Real)0.5;
    const int bo = threadIdx.x + 2;
    Real own_sum = (Real)0;  // FP64: the node's f summed; phi once the 1 / r table is filled
    if (inside) {
        if constexpr (sizeof(PT) == 2) {
            sphi[(threadIdx.y + 2) * LD + bo] = phi_of<Codec>(f0raw, fraw, rcp_(r), sa_of(j));
        } else {
            Real sum = (Real)f0_value(f0raw);
#pragma unroll
            for (int i = 1; i < 9; ++i) sum += Codec::dec_f(fraw[i - 1], (Real)w_of(i) * r);
            if constexpr (kInvrTable) own_sum = sum;
            else sphi[(threadIdx.y + 2) * LD + bo] = sum * rcp_(r);
        }
    } else {
        const int jm = ghost_r(j, g.nr);
        sphi[(threadIdx.y + 2) * LD + bo] = phi_of<Codec>(f0raw, fraw, rcp_((Real)jm + (Real)0.5), sa_of(jm));
    }
    // FP64: the node's moments while other warps still wait for their loads
    // (19.67 against 19.99 ms on the 512-case batch, bit-identical; in FP32
    // and bfloat16 storage the same was slower, 0.796 against 0.735 ms and
    // 0.761 against 0.735 ms)
    constexpr bool kPreEarly = sizeof(Real) == 8;
    PreCollision<Real> pre;
    if constexpr (kPreEarly) {
        if (inside) node_pre<Codec>(f0raw, fraw, graw, r, pre, nullptr, GridCol{});
    }
    // 3. the column tables and the case record into shared memory
    if constexpr (kInvrTable) {
        if (q < LD) s_invr[q] = (Real)1 / ((Real)(g.j0 - 2 + q) + (Real)0.5);
    }
    if constexpr (kG) {
        if (q < LD) grid_tab_fill<Codec>(T, q, g.j0, g.nr);
    }
    if (q < kCW) reinterpret_cast<int32_t*>(&sC)[q] = cw;
    if constexpr (kInvrTable) {
        // FP64: one division per column, not per node (a division is a long
        // sequence on the FP64 pipe), so the own phi waits for the table
        __syncthreads();
        if (inside) sphi[(threadIdx.y + 2) * LD + bo] = own_sum * s_invr[bo];
    }
    __syncthreads();
    if (!inside) return;
    const CaseDev& C = sC;
    const CaseView<Codec> V = case_view<Codec>(S, C);
    const int loc = k * C.pitch + j;
    // the lagged pressure p^{n-1}, read only under the lagged coupling
    if (C.p_coupling == 1) p_prev = V.in_node(loc).p();
    // 16-bit storage: the decoded f_0..8 go to the update (measured -1.5 %
    // against decoding them there; +0.6 % in FP32, where decoding is free)
    constexpr bool kKeepF = sizeof(PT) == 2;
    Real f[9];
    if constexpr (kKeepF) {
        f[0] = (Real)f0_value(f0raw);
        if constexpr (kG) {
            const GridCol gc = T.col(bo);
#pragma unroll
            for (int i = 1; i < 9; ++i) f[i] = Codec::dec_f(fraw[i - 1], gc, i > 4);
        } else {
#pragma unroll
            for (int i = 1; i < 9; ++i) f[i] = Codec::dec_f(fraw[i - 1], (Real)w_of(i) * r);
        }
    }

    if constexpr (kG) {
        const TabCols cols{T, j == 0 ? bo : bo - 1, bo, j + 1 == C.nr ? bo : bo + 1};
        node_update_grid<Codec, RM, LD>(C, V, sphi, threadIdx.y + 2, bo, k, j, loc, f0raw, fraw, graw, chz_prev,
                                        chr_prev, p_prev, f, cols);
    } else {
        if constexpr (kPreEarly) {
            node_update_pre<Codec, RM, LD>(C, V, sphi, threadIdx.y + 2, bo, k, j, loc, pre, chz_prev, chr_prev,
                                           p_prev, kInvrTable ? s_invr : nullptr, NoCols{});
        } else {
            node_update<Codec, RM, LD>(C, V, sphi, threadIdx.y + 2, bo, k, j, loc, f0raw, fraw, graw, chz_prev,
                                       chr_prev, p_prev, kInvrTable ? s_invr : nullptr, kKeepF ? f : nullptr,
                                       NoCols{});
        }
    }
}

// The step with two nodes per thread, one after the other: thread (x, y) of
// a CTA of BZ warps updates nodes (k0 + y, j0 + x) and (k0 + y + BZ, j0 + x)
// of a tile of 2 BZ rows with the one-node update of node_update, so the
// results are those of step_kernel.  Both nodes' loads are in flight before
// the tile's barrier (twice the loads per thread), and the phi ring is shared
// by twice the nodes.
//
// STASH: the second node's stored inputs wait in shared memory, not in
// registers, while the first node is updated, so the kernel fits fewer
// registers and more CTAs per SM (AXILBM_STASH_CTAS).
#ifndef AXILBM_SEQ2_CTAS
#define AXILBM_SEQ2_CTAS 3
#endif
#ifndef AXILBM_STASH_CTAS
#define AXILBM_STASH_CTAS 4
#endif
template <class Codec, int BZ, int RM, bool STASH = false>
constexpr int seq2_min_blocks() {
    return sizeof(typename Codec::Real) == 8
               ? 1
               : (STASH ? AXILBM_STASH_CTAS : (BZ >= 8 ? AXILBM_SEQ2_CTAS : 2 * AXILBM_SEQ2_CTAS));
}

template <class Codec, int BZ, int RM, bool STASH = false>
__global__ void __launch_bounds__(kTR * BZ, (seq2_min_blocks<Codec, BZ, RM, STASH>()))
step_kernel_seq2(const CaseDev* __restrict__ cases, const TileDev* __restrict__ tiles, StateDev<Codec> S,
                 const CUtensorMap* __restrict__ maps, int map_set, int parity, int ntiles, int ahead) {
    using Real = typename Codec::Real;
    using PT = typename Codec::PT;
    using PT2 = typename Codec::PT2;
    using F0T = typename Codec::F0T;
    constexpr int TZ = 2 * BZ;
    constexpr int NS = STASH ? kTR * BZ : 1;
    __shared__ F0T st_f0[NS];
    __shared__ PT2 st_pr[8][NS];
    __shared__ PT st_g0[NS];
    __shared__ Real st_chz[NS], st_chr[NS];
    constexpr int LD = kTR + 4;
    constexpr int NRING = 4 * kTR + 4 * (TZ + 4);
    static_assert(NRING == (TZ + 4) * LD - TZ * kTR, "the ring is the window without the tile");
    static_assert(sizeof(Real) == 4, "FP32 arithmetic");
    __shared__ Real sphi[(TZ + 4) * LD];
    __shared__ __align__(16) CaseDev sC;
    static_assert(sizeof(CaseDev) % 4 == 0 && sizeof(CaseDev) / 4 <= kTR * BZ, "one word per thread");
    constexpr bool kG = Codec::kGrid;
    __shared__ float4 sgA[kG ? LD : 1], sgD[kG ? LD : 1];
    __shared__ uint4 sgH[kG ? LD : 1];
    const GridTab T{sgA, sgD, sgH};
    const TileGeo g = reinterpret_cast<const TileGeo*>(tiles + ntiles)[blockIdx.x];
    const int q = threadIdx.y * kTR + threadIdx.x;
    constexpr int kCW = (int)(sizeof(CaseDev) / 4);  // words of the case record
    static_assert(NRING <= kTR * BZ, "one ring cell per thread at most");
    constexpr int kB = Block<Codec>::bytes;
    // 1. every global load of the window phase leaves before any of them is
    //    used, addressed from the tile's TileGeo record alone: this thread's
    //    word of the case record, both nodes' own values (out of the domain:
    //    the ghost node's f) and the f of this thread's ring cell
    int32_t cw = 0;
    if (q < kCW) cw = reinterpret_cast<const int32_t*>(cases + g.c)[q];
    if (maps != nullptr && q == 0 && (int)blockIdx.x + ahead < ntiles) {
        const TileDev tp = tiles[blockIdx.x + ahead];
        const CUtensorMap* M = maps + ((size_t)tp.c * 2 + map_set) * kMapsPerCase + 2 + parity;
        tensormap_acquire(M);
        tma_prefetch_4d(M, 0, 0, tp.j0 >> 5, tp.k0);
    }
    unsigned char* const base = const_cast<unsigned char*>(S.in) + (int64_t)g.blk0 * kB;  // the case's first block
    auto node_at = [&](int kk, int jj) { return Node<Codec>{base + (int64_t)(kk * g.rowblk + (jj >> 5)) * kB, jj & 31}; };
    const int j = g.j0 + threadIdx.x;
    F0T f0raw[2] = {};
    PT fraw[2][8], graw[2][9];
    Real chz_prev[2] = {}, chr_prev[2] = {}, p_prev[2] = {};
    bool in[2];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int k = g.k0 + threadIdx.y + p * BZ;
        in[p] = (j < g.nr) && (k < g.nz);
        if (in[p]) {
            const Node<Codec> n = node_at(k, j);
            f0raw[p] = n.f0();
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                const typename Codec::PT2 pr = n.pair(i);
                fraw[p][i - 1] = pr.x;
                graw[p][i] = pr.y;
            }
            graw[p][0] = n.g(0);
            chz_prev[p] = n.chz();
            chr_prev[p] = n.chr();
        } else {
            load_phi_raw<Codec>(node_at(ghost_z(k, g.nz, g.zper), ghost_r(j, g.nr)), f0raw[p], fraw[p]);
        }
    }
    // 2. the window: this thread's ring cell, then both nodes' own phi (Eq.
    //    16, in the form of the one-node kernel), as soon as their loads land;
    //    16-bit grid storage takes S_a of a column from grid_sa, the value the
    //    column table holds
    auto sa_of = [&](int jj) -> float {
        if constexpr (kG) return grid_sa<Codec>(jj);
        else return 0.0f;
    };
    if (q < NRING) {
        int ra, rb;
        ring_cell<TZ>(q, ra, rb);
        const int rj = ghost_r(g.j0 - 2 + rb, g.nr);
        F0T rf0;
        PT rf[8];
        load_phi_raw<Codec>(node_at(ghost_z(g.k0 - 2 + ra, g.nz, g.zper), rj), rf0, rf);
        sphi[ra * LD + rb] = phi_of<Codec>(rf0, rf, rcp_((Real)rj + (Real)0.5), sa_of(rj));
    }
    const Real r = (Real)j + (Real)0.5;
    const int bo = threadIdx.x + 2;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int a = threadIdx.y + 2 + p * BZ;
        if (in[p]) {
            if constexpr (sizeof(PT) == 2) {
                sphi[a * LD + bo] = phi_of<Codec>(f0raw[p], fraw[p], rcp_(r), sa_of(j));
            } else {
                Real sum = (Real)f0_value(f0raw[p]);
#pragma unroll
                for (int i = 1; i < 9; ++i) sum += Codec::dec_f(fraw[p][i - 1], (Real)w_of(i) * r);
                sphi[a * LD + bo] = sum * rcp_(r);
            }
        } else {
            const int jm = ghost_r(j, g.nr);
            sphi[a * LD + bo] = phi_of<Codec>(f0raw[p], fraw[p], rcp_((Real)jm + (Real)0.5), sa_of(jm));
        }
    }
    // 3. the column table and the case record into shared memory
    if constexpr (kG) {
        if (q < LD) grid_tab_fill<Codec>(T, q, g.j0, g.nr);
    }
    if (q < kCW) reinterpret_cast<int32_t*>(&sC)[q] = cw;
    if constexpr (STASH) {
        // the second node's inputs to shared memory (one slot per thread)
        const int q = threadIdx.y * kTR + threadIdx.x;
        if (in[1]) {
            st_f0[q] = f0raw[1];
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                PT2 pr;
                pr.x = fraw[1][i - 1];
                pr.y = graw[1][i];
                st_pr[i - 1][q] = pr;
            }
            st_g0[q] = graw[1][0];
            st_chz[q] = chz_prev[1];
            st_chr[q] = chr_prev[1];
        }
    }
    __syncthreads();
    const CaseDev& C = sC;
    const CaseView<Codec> V = case_view<Codec>(S, C);
    // the lagged pressure p^{n-1}, read only under the lagged coupling
    if (C.p_coupling == 1) {
#pragma unroll
        for (int p = 0; p < 2; ++p)
            if (in[p]) p_prev[p] = V.in_node((g.k0 + threadIdx.y + p * BZ) * C.pitch + j).p();
    }
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        if (!in[p]) continue;
        const int k = g.k0 + threadIdx.y + p * BZ;
        if (STASH && p == 1) {
            // reloaded only now: the compiler may not hoist these shared loads
            // above the first node's update
            asm volatile("" ::: "memory");
            const int q = threadIdx.y * kTR + threadIdx.x;
            f0raw[1] = st_f0[q];
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                const PT2 pr = st_pr[i - 1][q];
                fraw[1][i - 1] = pr.x;
                graw[1][i] = pr.y;
            }
            graw[1][0] = st_g0[q];
            chz_prev[1] = st_chz[q];
            chr_prev[1] = st_chr[q];
        }
        if constexpr (kG) {
            const TabCols cols{T, j == 0 ? bo : bo - 1, bo, j + 1 == C.nr ? bo : bo + 1};
            node_update_grid<Codec, RM, LD>(C, V, sphi, threadIdx.y + 2 + p * BZ, bo, k, j, k * C.pitch + j,
                                            f0raw[p], fraw[p], graw[p], chz_prev[p], chr_prev[p], p_prev[p],
                                            nullptr, cols);
        } else {
            node_update<Codec, RM, LD>(C, V, sphi, threadIdx.y + 2 + p * BZ, bo, k, j, k * C.pitch + j, f0raw[p],
                                       fraw[p], graw[p], chz_prev[p], chr_prev[p], p_prev[p], nullptr, nullptr,
                                       NoCols{});
        }
    }
}

// The packed update of the two nodes (k0, j) and (k0 + 8, j) of one thread
// of step_kernel_pack2, in two parts: pack2_moments decodes both nodes and
// transforms them in node pairs; pack2_finish runs the macroscopic step and
// both collisions in float2 lanes, then each node's inverse transform and
// stores.  Measured on the 512-case batch, against 0.657 ms in
// step_kernel_pack2 at the time: staging the tiles of this update through
// shared memory with the TMA pipeline of step_kernel_pipe (80 registers, 136
// bytes of spill) took 1.16 ms; a persistent kernel with one TMA stage
// refilled after the window barrier took 0.721 ms at 2 CTAs per SM (128
// registers) and 0.797 ms at 3 (160 bytes of spill).
//
// Step 4: M f and M g of (node 0, node 1) by the packed transforms of the
// one-node kernels (there they pair (f_i, g_i) of one node; each lane takes
// the same operations either way).  go: the constants of the nodes' column.
template <class Codec>
__device__ __forceinline__ void pack2_moments(const GridCol& go, const typename Codec::F0T* f0raw,
                                              const typename Codec::PT (*fraw)[8], const typename Codec::PT (*graw)[9],
                                              float2* mf, float2* mg, float2& g0) {
    float2 x[9];
    x[0] = make_float2(f0raw[0], f0raw[1]);
#pragma unroll
    for (int i = 1; i < 9; ++i)
        x[i] = make_float2(Codec::dec_f(fraw[0][i - 1], go, i > 4), Codec::dec_f(fraw[1][i - 1], go, i > 4));
    moments_p(x, mf);
    x[0] = make_float2(Codec::dec_g0(graw[0][0], go), Codec::dec_g0(graw[1][0], go));
    g0 = x[0];
#pragma unroll
    for (int i = 1; i < 9; ++i)
        x[i] = make_float2(Codec::dec_g(graw[0][i], go, i > 4), Codec::dec_g(graw[1][i], go, i > 4));
    moments_p(x, mg);
}

// Steps 5 and 6, from the moments of both nodes (the first node inside the
// case; in1: the second too) and the row-pair phi window.
template <class Codec, int RM, int LD>
__device__ __forceinline__ void pack2_finish(const CaseDev& C, const CaseView<Codec>& V, const float2* spair,
                                             const GridTab& T, int ty, int j, int k0, const float2* mf,
                                             const float2* mg, float2 g0, const float* chz_prev,
                                             const float* chr_prev, const float* p_prev, bool in1) {
    constexpr int BZ = 8;
    const int bo = (j & 31) + 2;  // the window column of j (tiles start at multiples of 32)
    const TabCols cols{T, j == 0 ? bo : bo - 1, bo, j + 1 == C.nr ? bo : bo + 1};
    // 5. the macroscopic step and both collisions once for both nodes
    lane::Macro<float2> m;
    lane::node_macros<float2, LD, RM, true>(C, spair, ty + 2, bo, j, mg, g0,
                                            make_float2(p_prev[0], p_prev[1]), m);
    float2 mpf[9], mpg[9], chz, chr;
    lane::collide_f<float2, RM>(C, m, mf, make_float2(chz_prev[0], chz_prev[1]),
                                make_float2(chr_prev[0], chr_prev[1]), chz, chr, mpf);
    lane::collide_g<float2, RM>(C, m, mpg);
    // 6. each node's populations (the (f_i, g_i)-paired inverse transform of
    //    the one-node kernels; measured faster here than transforming node
    //    pairs, 0.670 against 0.695 ms) and stores
    float mpf_n[9], mpg_n[9], fp[9], gp[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        mpf_n[i] = mpf[i].x;
        mpg_n[i] = mpg[i].x;
    }
    inverse_moments_fg(mpf_n, mpg_n, fp, gp);
    node_post_grid<Codec>(C, V, k0, j, k0 * C.pitch + j, fp, gp, chz.x, chr.x, m.p.x, mf[0].x, cols);
    if (in1) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            mpf_n[i] = mpf[i].y;
            mpg_n[i] = mpg[i].y;
        }
        inverse_moments_fg(mpf_n, mpg_n, fp, gp);
        const int k1 = k0 + BZ;
        node_post_grid<Codec>(C, V, k1, j, k1 * C.pitch + j, fp, gp, chz.y, chr.y, m.p.y, mf[0].y, cols);
    }
}

// The FP16 step with two nodes per thread in packed lanes (launch variant 7):
// thread (x, y) of an 8-warp CTA holds the nodes (k0 + y, j) and (k0 + y + 8,
// j) of a 16-row tile, decodes and stores each on its own, and runs the
// macroscopic step and both collisions once for both, in the float2 lanes of
// lbm_lane.cuh (one packed instruction per operation pair; the column's r,
// 1/r and case parameters shared).  The phi window is held as row pairs,
// spair[a][b] = (phi of window row a, of window row a + 8), so each stencil
// point of both nodes is one 8-byte shared load.  Every lane computes exactly
// what node_update_grid computes.
// The loads of the window phase are addressed from the tile's TileGeo record
// alone and all leave before any of them is used: the case record (one word
// per thread), both nodes' own values and the thread's ring cell.  The table
// and the case record are stored while they are in flight, and one barrier
// closes the window; both nodes' moments are formed before it.  Measured on
// the 512-case batch, before the moments moved ahead of the barrier and the
// FP32 approximations flushed subnormals (0.572 ms with both): 0.600 ms,
// against 0.658 ms when the case record was fetched and stored first (a
// barrier before the own and ring loads) and 0.688 ms with the geometry
// record but the case record fetched after the ring's loads were consumed.
// 3 CTAs per SM (80 registers, 20 bytes of spill); on the current build 2
// CTAs (no spill) take 0.664 ms and 4 take 0.596 ms.
#ifndef AXILBM_PACK2_CTAS
#define AXILBM_PACK2_CTAS 3
#endif

template <class Codec, int RM>
__global__ void __launch_bounds__(kTR * 8, AXILBM_PACK2_CTAS)
step_kernel_pack2(const CaseDev* __restrict__ cases, const TileGeo* __restrict__ geo, StateDev<Codec> S,
                  const CUtensorMap* __restrict__ maps, int parity, int ntiles, int ahead) {
    static_assert(Codec::kGrid, "the FP16 grid codec's packed step");
    using PT = typename Codec::PT;
    using F0T = typename Codec::F0T;
    constexpr int BZ = 8, TZ = 2 * BZ, LD = kTR + 4, NP = BZ + 4;
    constexpr int NRING = 4 * kTR + 4 * (TZ + 4);
    static_assert(NRING <= kTR * BZ, "one ring cell per thread at most");
    constexpr int kB = Block<Codec>::bytes;
    __shared__ float2 spair[NP * LD];
    __shared__ __align__(16) CaseDev sC;
    __shared__ float4 sgA[LD], sgD[LD];
    __shared__ uint4 sgH[LD];
    const GridTab T{sgA, sgD, sgH};
    const TileGeo g = geo[blockIdx.x];
    const int q = threadIdx.y * kTR + threadIdx.x;
    constexpr int kCW = (int)(sizeof(CaseDev) / 4);  // words of the case record
    // 1. every load of the window phase is issued before any of them is used:
    //    the case record word of this thread, both nodes' own values and the
    //    raw values of this thread's ring cell
    int32_t cw = 0;
    if (q < kCW) cw = reinterpret_cast<const int32_t*>(cases + g.c)[q];
    if (maps != nullptr && q == 0 && (int)blockIdx.x + ahead < ntiles) {
        // L2 prefetch of the tile one resident wave ahead
        const TileGeo tp = geo[blockIdx.x + ahead];
        const CUtensorMap* M = maps + ((size_t)tp.c * 2 + 1) * kMapsPerCase + 2 + parity;
        tensormap_acquire(M);
        tma_prefetch_4d(M, 0, 0, tp.j0 >> 5, tp.k0);
    }
    unsigned char* const base = const_cast<unsigned char*>(S.in) + (int64_t)g.blk0 * kB;  // the case's first block
    const int j = g.j0 + threadIdx.x;
    F0T f0raw[2] = {};
    PT fraw[2][8], graw[2][9];
    float chz_prev[2] = {}, chr_prev[2] = {}, p_prev[2] = {};
    bool in[2];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int k = g.k0 + threadIdx.y + p * BZ;
        in[p] = (j < g.nr) && (k < g.nz);
        if (in[p]) {
            const Node<Codec> n{base + (int64_t)(k * g.rowblk + (j >> 5)) * kB, j & 31};
            f0raw[p] = n.f0();
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                const typename Codec::PT2 pr = n.pair(i);
                fraw[p][i - 1] = pr.x;
                graw[p][i] = pr.y;
            }
            graw[p][0] = n.g(0);
            chz_prev[p] = n.chz();
            chr_prev[p] = n.chr();
        }
    }
    int ra = 0, rb = 0, rj = 0;
    F0T rf0 = {};
    PT rf[8];
    if (q < NRING) {
        ring_cell<TZ>(q, ra, rb);
        const int km = ghost_z(g.k0 - 2 + ra, g.nz, g.zper);
        rj = ghost_r(g.j0 - 2 + rb, g.nr);
        const Node<Codec> n{base + (int64_t)(km * g.rowblk + (rj >> 5)) * kB, rj & 31};
        rf0 = n.f0();
#pragma unroll
        for (int i = 1; i < 9; ++i) rf[i - 1] = n.f(i);
    }
    // 2. the column table and the case record into shared memory
    // (the table by the last 36 threads, which have no ring cell: 0.569
    // against 0.572 ms when the first 36 filled it)
    static_assert(NRING + LD <= kTR * BZ, "table threads without a ring cell");
    if (q >= kTR * BZ - LD) grid_tab_fill<Codec>(T, q - (kTR * BZ - LD), g.j0, g.nr);
    if (q < kCW) reinterpret_cast<int32_t*>(&sC)[q] = cw;
    // 3. the window: the ring cell and both nodes' own phi
    auto put = [&](int a, int b, float v) {
        if (a < NP) spair[a * LD + b].x = v;
        if (a >= BZ) spair[(a - BZ) * LD + b].y = v;
    };
    if (q < NRING) put(ra, rb, phi_of<Codec>(rf0, rf, rcp_((float)rj + 0.5f), grid_sa<Codec>(rj)));
    const float r = (float)j + 0.5f;
    const int bo = threadIdx.x + 2;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int a = threadIdx.y + 2 + p * BZ;
        if (in[p]) {
            put(a, bo, phi_of<Codec>(f0raw[p], fraw[p], rcp_(r), grid_sa<Codec>(j)));
        } else {
            const int km = ghost_z(g.k0 + threadIdx.y + p * BZ, g.nz, g.zper);
            const int jm = ghost_r(j, g.nr);
            const Node<Codec> n{base + (int64_t)(km * g.rowblk + (jm >> 5)) * kB, jm & 31};
            put(a, bo, node_phi<Codec>(n, rcp_((float)jm + 0.5f), grid_sa<Codec>(jm)));
        }
    }
    // 4. both nodes' moments while other warps still wait for their loads
    //    (the column's constants computed, as the table holds them).
    //    Measured against forming them after the barrier: 0.572 against
    //    0.580 ms, and 0.598 against 0.646 ms with raw moments
    float2 mf[9], mg[9], g0;
    pack2_moments<Codec>(grid_col<Codec>(j), f0raw, fraw, graw, mf, mg, g0);
    __syncthreads();
    if (!in[0]) return;  // the second node lies below the first
    const CaseDev& C = sC;
    const CaseView<Codec> V = case_view<Codec>(S, C);
    // the lagged pressure p^{n-1}, read only under the lagged coupling (a flag
    // of the case record)
    if (C.p_coupling == 1) {
#pragma unroll
        for (int p = 0; p < 2; ++p)
            if (in[p]) p_prev[p] = V.in_node((g.k0 + threadIdx.y + p * BZ) * C.pitch + j).p();
    }
    pack2_finish<Codec, RM, LD>(C, V, spair, T, threadIdx.y, j, g.k0 + threadIdx.y, mf, mg, g0, chz_prev, chr_prev,
                                p_prev, in[1]);
}

// Shared-memory layout of one stage of the TMA-pipelined step for tile
// height TZ, then the phi window and one mbarrier per stage.  A stage holds
// its tile's record, the record of the tile after it in the CTA's walk, the
// tile's case record and the storage blocks of the tile's column group for
// rows k0-2 .. k0+TZ+1 (the tile plus the rows of the phi window's ring; rows
// outside the case read as zero and are never used).
template <class Codec, int TZ>
struct TmaTile {
    using Real = typename Codec::Real;
    static constexpr int HR = TZ + 4;          // rows k0-2 .. k0+TZ+1
    static constexpr int LD = kTR + 4;         // phi window row length
    static constexpr size_t al(size_t b) { return (b + 127) / 128 * 128; }
    static constexpr size_t box_bytes = (size_t)HR * Block<Codec>::bytes;
    // offsets inside one stage
    static constexpr size_t off_rec = 0;                   // TileDev of this stage's tile
    static constexpr size_t off_next = 16;                 // TileDev of the CTA's next tile after it
    static constexpr size_t off_case = 32;                 // CaseDev of the tile's case
    static constexpr size_t off_box = al(off_case + sizeof(CaseDev));
    static constexpr size_t stage_bytes = al(off_box + box_bytes);
    // two stages when they fit, else one (FP64 with tall tiles)
    static constexpr int NS = (2 * stage_bytes + 16384 <= 200 * 1024) ? 2 : 1;
    static constexpr size_t off_phi = NS * stage_bytes;
    static constexpr size_t off_bar = al(off_phi + (size_t)HR * LD * sizeof(Real));
    static constexpr size_t bytes = off_bar + 128;
};

// Fill one stage with tile `tt` (whose successor in the CTA's walk is tile
// index `next`): records, case record and one tensor copy of the blocks, all
// completing on `bar`.  Called by one thread.
template <class Codec, int BZ>
__device__ __forceinline__ void tma_issue(unsigned char* stage, const TileDev tt, int next, int ntiles,
                                          const CaseDev* cases, const TileDev* tiles, const CUtensorMap* maps,
                                          int map_set, int parity, uint64_t* bar) {
    using L = TmaTile<Codec, BZ>;
    *(TileDev*)(stage + L::off_rec) = tt;
    const CUtensorMap* M = maps + ((size_t)tt.c * 2 + map_set) * kMapsPerCase + parity;
    tensormap_acquire(M);
    const bool has_next = next < ntiles;
    mbar_expect_tx(bar, (uint32_t)L::box_bytes + (uint32_t)sizeof(CaseDev) + (has_next ? (uint32_t)sizeof(TileDev) : 0u));
    bulk_load(stage + L::off_case, cases + tt.c, (uint32_t)sizeof(CaseDev), bar);
    if (has_next) bulk_load(stage + L::off_next, tiles + next, (uint32_t)sizeof(TileDev), bar);
    // dims: 32 words, 128-byte slots of a block, column groups, rows
    tma_load_4d(stage + L::off_box, M, 0, 0, tt.j0 >> 5, tt.k0 - 2, bar);
}

// phi at window cell (a, b) of tile tt (Eq. 16 + ghost rules), from the
// staged blocks when the ghost-mapped node lies in the tile's column group and
// the staged rows, else from global memory.
template <class Codec, int TZ>
__device__ __forceinline__ typename Codec::Real staged_phi(const unsigned char* st, const CaseDev& C,
                                                           const CaseView<Codec>& V, const TileDev& tt, int a,
                                                           int b) {
    using L = TmaTile<Codec, TZ>;
    using Real = typename Codec::Real;
    const int km = ghost_z(tt.k0 - 2 + a, C.nz, C.zper);
    const int jm = ghost_r(tt.j0 - 2 + b, C.nr);
    const int sa = km - (tt.k0 - 2);
    const Real r = (Real)jm + (Real)0.5;
    float Sa = 0.0f;
    if constexpr (Codec::kGrid) Sa = grid_sa<Codec>(jm);
    if (sa >= 0 && sa < L::HR && (jm >> 5) == (tt.j0 >> 5)) {
        const Node<Codec> n{const_cast<unsigned char*>(st + L::off_box) + (size_t)sa * Block<Codec>::bytes, jm & 31};
        return node_phi<Codec>(n, rcp_(r), Sa);
    }
    return node_phi<Codec>(V.in_node(km * C.pitch + jm), rcp_(r), Sa);
}

// Resident CTAs per SM: as many as the stages' shared memory allows (up to
// 227 KB per SM, 1 KB reserved per CTA), at most 3 of 256 threads (80
// registers a thread, which the pipelined loop needs to stay clear of spills)
// or 2 of 512; one for FP64.
template <class Codec, int BZ>
constexpr int pipe_min_blocks() {
    constexpr int by_smem = (int)((227u * 1024u) / (TmaTile<Codec, BZ>::bytes + 1024u));
    constexpr int by_regs = BZ >= 16 ? 2 : 3;
    return sizeof(typename Codec::Real) == 8 ? 1 : (by_smem < 1 ? 1 : (by_smem < by_regs ? by_smem : by_regs));
}

// The same step as step_kernel, with each tile's inputs staged in shared
// memory by TMA, persistent and pipelined.  Each CTA walks the tile list with
// stride gridDim.x.  After the copies of tile n have landed, one thread issues
// those of tile n+1 into the other stage (the tile's record came with tile
// n's stage), so they overlap the work on tile n; no thread ever waits on a
// global load before its tile's data is in shared memory.  Each node's own phi
// comes from its staged populations; the ring of the phi window is summed from
// the staged box.  Every thread waits on the stage's mbarrier with a bounded
// number of tries.  A timeout sets the status word; the timed-out stage gets a
// second bounded wait and the CTA leaves.  Nothing else of its own is in
// flight then, since the next stage is issued only after a successful wait.
template <class Codec, int BZ, int RM>
__global__ void __launch_bounds__(kTR * BZ, (pipe_min_blocks<Codec, BZ>()))
step_kernel_pipe(const CaseDev* __restrict__ cases, const TileDev* __restrict__ tiles, int ntiles,
                 StateDev<Codec> S, const CUtensorMap* __restrict__ maps, int map_set, int parity,
                 int* __restrict__ status) {
    using Real = typename Codec::Real;
    using PT = typename Codec::PT;
    using F0T = typename Codec::F0T;
    using L = TmaTile<Codec, BZ>;
    constexpr int TZ = BZ, LD = L::LD, NS = L::NS;
    constexpr int NRING = 4 * kTR + 4 * (TZ + 4);
    static_assert(NRING == (TZ + 4) * LD - TZ * kTR, "the ring is the window without the tile");
    constexpr int kWaitTries = 1 << 22;
    extern __shared__ __align__(128) unsigned char smem[];
    Real* sphi = (Real*)(smem + L::off_phi);  // [HR][LD]
    uint64_t* bar = (uint64_t*)(smem + L::off_bar);
    const int tid = threadIdx.y * kTR + threadIdx.x;
    if ((int)blockIdx.x >= ntiles) return;
    if (tid == 0) {
        for (int q = 0; q < NS; ++q) mbar_init(bar + q, 1);
    }
    __syncthreads();
    if (tid == 0)
        tma_issue<Codec, BZ>(smem, tiles[blockIdx.x], blockIdx.x + gridDim.x, ntiles, cases, tiles, maps, map_set,
                             parity, bar);
    unsigned phases = 0u;  // bit s: parity of the next phase of stage s
    for (int n = 0, t = blockIdx.x; t < ntiles; ++n, t += gridDim.x) {
        const int s = NS == 2 ? (n & 1) : 0;
        const unsigned char* st = smem + s * L::stage_bytes;
        // this barrier also closes every read of the other stage and of the
        // phi window made while working on the previous tile
        const unsigned ph = (phases >> s) & 1u;
        const bool ok = __syncthreads_and(mbar_wait_bounded(bar + s, ph, status, kWaitTries));
        if (!ok) {
            // this stage's copies get a second bounded chance to land before the CTA leaves
            if (tid == 0) mbar_wait_bounded(bar + s, ph, status, kWaitTries);
            __syncthreads();
            return;
        }
        phases ^= 1u << s;
        const int tn = t + gridDim.x;
        if (NS == 2 && tid == 0 && tn < ntiles) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tma_issue<Codec, BZ>(smem + (s ^ 1) * L::stage_bytes, *(const TileDev*)(st + L::off_next),
                                 tn + gridDim.x, ntiles, cases, tiles, maps, map_set, parity, bar + (s ^ 1));
        }
        const TileDev tt = *(const TileDev*)(st + L::off_rec);
        const CaseDev& C = *(const CaseDev*)(st + L::off_case);
        const CaseView<Codec> V = case_view<Codec>(S, C);
        const int j = tt.j0 + threadIdx.x;
        const int k = tt.k0 + threadIdx.y;
        const bool inside = (j < C.nr) && (k < C.nz);
        // own staged inputs: block of row ty + 2 of the box, lane tx
        F0T f0raw{};
        PT fraw[8], graw[9];
        Real chz_prev = (Real)0, chr_prev = (Real)0, p_prev = (Real)0;
        if (inside) {
            const Node<Codec> n{const_cast<unsigned char*>(st + L::off_box) +
                                    (size_t)(threadIdx.y + 2) * Block<Codec>::bytes,
                                (int)threadIdx.x};
            f0raw = n.f0();
#pragma unroll
            for (int i = 1; i < 9; ++i) fraw[i - 1] = n.f(i);
#pragma unroll
            for (int i = 0; i < 9; ++i) graw[i] = n.g(i);
            chz_prev = n.chz();
            chr_prev = n.chr();
            if (C.p_coupling == 1) p_prev = n.p();
        }
        // the ring of the phi window, from the staged box
        for (int q = tid; q < NRING; q += kTR * BZ) {
            int a, b;
            ring_cell<TZ>(q, a, b);
            sphi[a * LD + b] = staged_phi<Codec, TZ>(st, C, V, tt, a, b);
        }
        // the node's own phi (Eq. 16) from its staged populations
        const Real r = (Real)j + (Real)0.5;
        Real f[9];
        if (inside) {
            if constexpr (Codec::kGrid) {
                const GridCol g = grid_col<Codec>(j);
                f[0] = f0_value(f0raw);
#pragma unroll
                for (int i = 1; i < 9; ++i) f[i] = Codec::dec_f(fraw[i - 1], g, i > 4);
                sphi[(threadIdx.y + 2) * LD + threadIdx.x + 2] = phi_of<Codec>(f0raw, fraw, rcp_(r), g.S_a);
            } else {
                f[0] = (Real)f0_value(f0raw);
                Real sum = f[0];
#pragma unroll
                for (int i = 1; i < 9; ++i) {
                    f[i] = Codec::dec_f(fraw[i - 1], (Real)w_of(i) * r);
                    sum += f[i];
                }
                sphi[(threadIdx.y + 2) * LD + threadIdx.x + 2] =
                    sizeof(PT) == 2 ? phi_of<Codec>(f0raw, fraw, rcp_(r)) : sum * rcp_(r);
            }
        } else {
            sphi[(threadIdx.y + 2) * LD + threadIdx.x + 2] =
                staged_phi<Codec, TZ>(st, C, V, tt, threadIdx.y + 2, threadIdx.x + 2);
        }
        __syncthreads();
        if (inside) {
            const int loc = k * C.pitch + j;
            if constexpr (Codec::kGrid) {
                const CalcCols<Codec> cols{j == 0 ? j : j - 1, j, j + 1 == C.nr ? j : j + 1};
                node_update_grid<Codec, RM, LD>(C, V, sphi, threadIdx.y + 2, threadIdx.x + 2, k, j, loc, f0raw,
                                                fraw, graw, chz_prev, chr_prev, p_prev, f, cols);
            } else {
                node_update<Codec, RM, LD>(C, V, sphi, threadIdx.y + 2, threadIdx.x + 2, k, j, loc, f0raw, fraw,
                                           graw, chz_prev, chr_prev, p_prev, nullptr,
                                           sizeof(PT) == 2 ? f : nullptr, NoCols{});
            }
        }
        if (NS == 1) {
            // every read of the single stage is done before it is refilled
            __syncthreads();
            if (tid == 0 && tn < ntiles) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                tma_issue<Codec, BZ>(smem, *(const TileDev*)(st + L::off_next), tn + gridDim.x, ntiles, cases,
                                     tiles, maps, map_set, parity, bar);
            }
        }
    }
}

// phi, rho, u_z, u_r, p of one case into dense FP64 arrays out[5][nz][nr].
template <class Codec>
__global__ void __launch_bounds__(kTR * 8)
fields_kernel(const CaseDev* __restrict__ cases, const TileDev* __restrict__ tiles, StateDev<Codec> S,
              double* __restrict__ out) {
    using Real = typename Codec::Real;
    constexpr int TZ = 8;
    constexpr int LD = kTR + 4;
    __shared__ Real sphi[(TZ + 4) * LD];
    const TileDev t = tiles[blockIdx.x];
    const CaseDev& C = cases[t.c];
    const CaseView<Codec> V = case_view<Codec>(S, C);
    for (int idx = threadIdx.y * kTR + threadIdx.x; idx < (TZ + 4) * LD; idx += kTR * 8)
        sphi[idx] = window_phi<Codec>(C, V, t, idx / LD, idx % LD);
    __syncthreads();
    const int j = t.j0 + threadIdx.x, k = t.k0 + threadIdx.y;
    if (j >= C.nr || k >= C.nz) return;
    const int loc = k * C.pitch + j;
    const Real r = (Real)j + (Real)0.5;
    const Node<Codec> nd = V.in_node(loc);
    Real g[9];
    if constexpr (Codec::kGrid) {
        const GridCol gc = grid_col<Codec>(j);
        g[0] = Codec::dec_g0(nd.g(0), gc);
#pragma unroll
        for (int i = 1; i < 9; ++i) g[i] = Codec::dec_g(nd.g(i), gc, i > 4);
    } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = Codec::dec_g(nd.g(i), (Real)w_of(i) * r);
    }
    Macro<Real> m;
    Real mg[9];
    moments<Real>(g, mg);
    node_macros<Real, LD>(C, sphi, threadIdx.y + 2, threadIdx.x + 2, j, mg, g[0], C.p_coupling == 1 ? nd.p() : (Real)0,
                          m);
    const int64_t n = (int64_t)C.nz * C.nr, o = (int64_t)k * C.nr + j;
    out[o] = (double)m.phi;
    out[n + o] = (double)m.rho;
    out[2 * n + o] = (double)m.uz;
    out[3 * n + o] = (double)m.ur;
    out[4 * n + o] = (double)m.p;
}

// Initial condition of node (k, j) of case C from its phi0 (Eq. 11): f =
// f^eq(phi0, u = 0), g = 0, chi^{-1} = (0, M phi0), p^{-1} = 0, written to the
// "in" buffers.
template <class Codec>
__device__ __forceinline__ void init_node(const CaseDev& C, const StateDev<Codec>& S, int k, int j, double phi0) {
    using Real = typename Codec::Real;
    const CaseView<Codec> V = case_view<Codec>(S, C);
    const int loc = k * C.pitch + j;
    const Node<Codec> n = V.in_node(loc);
    const CaseReal<Real>& P = case_params<Real>(C);
    const Real phi = (Real)phi0;
    const Real r = (Real)j + (Real)0.5;
    Real fe[9];
    FF ledger{0.0f, 0.0f};
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        fe[i] = (Real)w_of(i) * (r * phi + (Real)cr_of(i) * P.mob * phi * (Real)3);
        if constexpr (Codec::kLedger) ff_add(ledger, (float)fe[i]);
    }
    if constexpr (Codec::kGrid) {
        // f_0 takes the rest of the node's total, rounded onto its ledger grid
        const GridCol g = grid_col<Codec>(j);
        float rest = 0.0f;
#pragma unroll
        for (int i = 0; i < 9; ++i) rest += fe[i];
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            const auto e = Codec::enc_f(fe[i], g, i > 4);
            n.f(i) = e;
            rest -= Codec::dec_f(e, g, i > 4);
        }
        n.f0() = grid_round_f0<Codec>(rest, j);
        n.g(0) = Codec::enc_g0((Real)0, g);
#pragma unroll
        for (int i = 1; i < 9; ++i) n.g(i) = Codec::enc_g((Real)0, g, i > 4);
    } else {
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            const Real wr = (Real)w_of(i) * r;
            const auto e = Codec::enc_f(fe[i], wr, (Real)1 / wr);
            n.f(i) = e;
            if constexpr (Codec::kLedger) ff_add(ledger, -(float)Codec::dec_f(e, wr));
        }
        if constexpr (Codec::kLedger) {
            const FF l = ff_norm(ledger);
            n.f0() = make_float2(l.hi, l.lo);
        } else {
            n.f0() = fe[0];
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) n.g(i) = Codec::enc_g((Real)0, (Real)w_of(i) * r, (Real)1);
    }
    n.chz() = (Real)0;
    n.chr() = P.mob * phi;
    n.p() = (Real)0;
}

// Initial condition of the cases of a tile list, one CTA per 8-row tile:
// node (k, j) of case c takes phi0[dense_off(c) - base + k nr + j], so one
// array may hold every case's dense [nz][nr] phi0 in case order (base 0), or
// one case's alone (base = that case's dense_off).
template <class Codec>
__global__ void __launch_bounds__(kTR * 8) init_kernel(const CaseDev* __restrict__ cases,
                                                       const TileDev* __restrict__ tiles,
                                                       const double* __restrict__ phi0, int64_t base,
                                                       StateDev<Codec> S) {
    const TileDev t = tiles[blockIdx.x];
    const CaseDev& C = cases[t.c];
    const int j = t.j0 + threadIdx.x, k = t.k0 + threadIdx.y;
    if (j >= C.nr || k >= C.nz) return;
    init_node<Codec>(C, S, k, j, phi0[C.dense_off - base + (int64_t)k * C.nr + j]);
}

// Decode the state of one case into FP64 arrays (f[9], g[9], aux[3], each [nz][nr]).
template <class Codec>
__global__ void get_state_kernel(CaseDev C, StateDev<Codec> S, double* f, double* g, double* aux) {
    using Real = typename Codec::Real;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (j >= C.nr || k >= C.nz) return;
    const CaseView<Codec> V = case_view<Codec>(S, C);
    const Node<Codec> nd = V.in_node(k * C.pitch + j);
    const int64_t n = (int64_t)C.nz * C.nr, o = (int64_t)k * C.nr + j;
    const Real r = (Real)j + (Real)0.5;
    if constexpr (Codec::kGrid) {
        const GridCol gc = grid_col<Codec>(j);
        if (f) {
            f[o] = (double)nd.f0();
            for (int i = 1; i < 9; ++i) f[i * n + o] = (double)Codec::dec_f(nd.f(i), gc, i > 4);
        }
        if (g) {
            g[o] = (double)Codec::dec_g0(nd.g(0), gc);
            for (int i = 1; i < 9; ++i) g[i * n + o] = (double)Codec::dec_g(nd.g(i), gc, i > 4);
        }
    } else {
        if (f) {
            if constexpr (Codec::kLedger) {
                const float2 v = nd.f0();
                f[o] = (double)v.x + (double)v.y;
            } else {
                f[o] = (double)f0_value(nd.f0());
            }
            for (int i = 1; i < 9; ++i) f[i * n + o] = (double)Codec::dec_f(nd.f(i), (Real)w_of(i) * r);
        }
        if (g) {
            for (int i = 0; i < 9; ++i) g[i * n + o] = (double)Codec::dec_g(nd.g(i), (Real)w_of(i) * r);
        }
    }
    if (aux) {
        aux[o] = (double)nd.chz();
        aux[n + o] = (double)nd.chr();
        aux[2 * n + o] = (double)nd.p();
    }
}

// Encode FP64 arrays into the current ("in") state buffers of one case.
template <class Codec>
__global__ void set_state_kernel(CaseDev C, StateDev<Codec> S, const double* f, const double* g, const double* aux) {
    using Real = typename Codec::Real;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (j >= C.nr || k >= C.nz) return;
    const CaseView<Codec> V = case_view<Codec>(S, C);
    const Node<Codec> nd = V.in_node(k * C.pitch + j);
    const int64_t n = (int64_t)C.nz * C.nr, o = (int64_t)k * C.nr + j;
    const Real r = (Real)j + (Real)0.5;
    if constexpr (Codec::kGrid) {
        const GridCol gc = grid_col<Codec>(j);
        if (f) {
            // f_0 = the given f_0 plus the rounding of f_1..8 (in FP64), on the
            // node's ledger grid: the stored populations sum to the input sum
            // up to that last rounding
            double v = f[o];
            for (int i = 1; i < 9; ++i) {
                const auto e = Codec::enc_f((float)f[i * n + o], gc, i > 4);
                nd.f(i) = e;
                v += f[i * n + o] - (double)Codec::dec_f(e, gc, i > 4);
            }
            // the ledger grid q = 2^-kGridExp ulp(S_5(max(j - 1, 0))) at kScaleBits bits
            int ex = 0;
            frexp((double)(0.25f * grid_sa<Codec>(max(j - 1, 0))), &ex);
            const double q = ldexp(1.0, ex - Codec::kScaleBits - Codec::kGridExp);
            nd.f0() = (float)(rint(v / q) * q);
        }
        if (g) {
            nd.g(0) = Codec::enc_g0((float)g[o], gc);
            for (int i = 1; i < 9; ++i) nd.g(i) = Codec::enc_g((float)g[i * n + o], gc, i > 4);
        }
    } else {
        if (f) {
            if constexpr (Codec::kLedger) {
                // ledger = f_0 exactly as given (split into a float pair) plus the
                // rounding of f_1..8, so the stored populations sum to the input sum
                const double v0 = f[o];
                FF ledger{(float)v0, (float)(v0 - (double)(float)v0)};
                for (int i = 1; i < 9; ++i) {
                    const Real wr = (Real)w_of(i) * r;
                    const auto e = Codec::enc_f((Real)f[i * n + o], wr, (Real)1 / wr);
                    nd.f(i) = e;
                    ff_add(ledger, (float)f[i * n + o]);
                    ff_add(ledger, (float)(f[i * n + o] - (double)(float)f[i * n + o]));
                    ff_add(ledger, -(float)Codec::dec_f(e, wr));
                }
                const FF l = ff_norm(ledger);
                *reinterpret_cast<float2*>(&nd.f0()) = make_float2(l.hi, l.lo);
            } else {
                for (int i = 1; i < 9; ++i) {
                    const Real wr = (Real)w_of(i) * r;
                    nd.f(i) = Codec::enc_f((Real)f[i * n + o], wr, (Real)1 / wr);
                }
                *reinterpret_cast<double*>(&nd.f0()) = f[o];
            }
        }
        if (g) {
            for (int i = 0; i < 9; ++i) {
                const Real wr = (Real)w_of(i) * r;
                nd.g(i) = Codec::enc_g((Real)g[i * n + o], wr, (Real)1 / wr);
            }
        }
    }
    if (aux) {
        nd.chz() = (Real)aux[o];
        nd.chr() = (Real)aux[n + o];
        nd.p() = (Real)aux[2 * n + o];
    }
}

// ---------------------------------------------------------------- host launchers
template <class Codec>
StateDev<Codec> make_state(const DeviceState& D, int parity) {
    static_assert(Block<Codec>::bytes == block_bytes_of((int)sizeof(typename Codec::F0T),
                                                        (int)sizeof(typename Codec::PT),
                                                        (int)sizeof(typename Codec::Real)),
                  "host and device block sizes");
    StateDev<Codec> S;
    const int a = parity & 1, b = a ^ 1;
    S.in = (const unsigned char*)D.blk[a];
    S.out = (unsigned char*)D.blk[b];
    return S;
}

// Persistent grid for the pipelined kernel: as many CTAs as fit on the GPU at
// once (queried per instantiation), capped by the tile count.
template <class Codec, int BZ, int RM>
void launch_tma(int ntiles, cudaStream_t st, const CaseDev* cs, const TileDev* tiles, const StateDev<Codec>& S,
                const DeviceState& D, int parity) {
    using L = TmaTile<Codec, BZ>;
    static int grid_cap = 0;
    if (grid_cap == 0) {
        cudaFuncSetAttribute(step_kernel_pipe<Codec, BZ, RM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes);
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_kernel_pipe<Codec, BZ, RM>, kTR * BZ, L::bytes);
        grid_cap = (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
    }
    const int grid = ntiles < grid_cap ? ntiles : grid_cap;
    step_kernel_pipe<Codec, BZ, RM><<<grid, dim3(kTR, BZ), L::bytes, st>>>(
        cs, tiles, ntiles, S, (const CUtensorMap*)D.tmaps, BZ == 8 ? 0 : 1, parity, D.status);
}

template <class Codec, int RM>
void launch_step_rates(int variant, int ntiles, cudaStream_t st, const CaseDev* cs, const TileDev* tiles,
                       const StateDev<Codec>& S, const DeviceState& D, int parity) {
    // prefetch distance: the CTAs resident at once (SMs x CTAs per SM)
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    const CUtensorMap* maps = (const CUtensorMap*)D.tmaps;
    switch (variant) {
        case 0:
            step_kernel<Codec, 8, RM><<<ntiles, dim3(kTR, 8), 0, st>>>(
                cs, tiles, S, maps, 0, parity, ntiles, kPrefetchQuarters * sms * step_min_blocks<Codec, 8, RM>() / 4);
            break;
        case 1:
            step_kernel<Codec, 16, RM><<<ntiles, dim3(kTR, 16), 0, st>>>(
                cs, tiles, S, maps, 1, parity, ntiles, kPrefetchQuarters * sms * step_min_blocks<Codec, 16, RM>() / 4);
            break;
        case 2:
            step_kernel<Codec, 4, RM><<<ntiles, dim3(kTR, 4), 0, st>>>(
                cs, tiles, S, maps, 0, parity, ntiles, kPrefetchQuarters * sms * step_min_blocks<Codec, 4, RM>() / 4);
            break;
        case 3: launch_tma<Codec, 8, RM>(ntiles, st, cs, tiles, S, D, parity); break;
        case 4: launch_tma<Codec, 16, RM>(ntiles, st, cs, tiles, S, D, parity); break;
        case 5:
            if constexpr (sizeof(typename Codec::Real) == 4)
                step_kernel_seq2<Codec, 8, RM><<<ntiles, dim3(kTR, 8), 0, st>>>(
                    cs, tiles, S, maps, 1, parity, ntiles, kPrefetchQuarters * sms * seq2_min_blocks<Codec, 8, RM>() / 4);
            else
                step_kernel<Codec, 16, RM><<<ntiles, dim3(kTR, 16), 0, st>>>(
                    cs, tiles, S, maps, 1, parity, ntiles, kPrefetchQuarters * sms * step_min_blocks<Codec, 16, RM>() / 4);
            break;
        case 7:
            if constexpr (Codec::kGrid)
                step_kernel_pack2<Codec, RM><<<ntiles, dim3(kTR, 8), 0, st>>>(
                    cs, reinterpret_cast<const TileGeo*>(tiles + ntiles), S, maps, parity, ntiles,
                    kPrefetchQuarters * sms * AXILBM_PACK2_CTAS / 4);
            else if constexpr (sizeof(typename Codec::Real) == 4)
                step_kernel_seq2<Codec, 8, RM><<<ntiles, dim3(kTR, 8), 0, st>>>(
                    cs, tiles, S, maps, 1, parity, ntiles, kPrefetchQuarters * sms * seq2_min_blocks<Codec, 8, RM>() / 4);
            else
                step_kernel<Codec, 16, RM><<<ntiles, dim3(kTR, 16), 0, st>>>(
                    cs, tiles, S, maps, 1, parity, ntiles, kPrefetchQuarters * sms * step_min_blocks<Codec, 16, RM>() / 4);
            break;
        default:
            if constexpr (sizeof(typename Codec::Real) == 4)
                step_kernel_seq2<Codec, 8, RM, true><<<ntiles, dim3(kTR, 8), 0, st>>>(
                    cs, tiles, S, maps, 1, parity, ntiles,
                    kPrefetchQuarters * sms * seq2_min_blocks<Codec, 8, RM, true>() / 4);
            else
                step_kernel<Codec, 16, RM><<<ntiles, dim3(kTR, 16), 0, st>>>(
                    cs, tiles, S, maps, 1, parity, ntiles, kPrefetchQuarters * sms * step_min_blocks<Codec, 16, RM>() / 4);
            break;
    }
}

template <class Codec>
cudaError_t launch_step_t(const DeviceState& D, int parity, int variant, const TileDev* tiles, int ntiles,
                          cudaStream_t st) {
    if (ntiles <= 0) return cudaSuccess;
    StateDev<Codec> S = make_state<Codec>(D, parity);
    const CaseDev* cs = (const CaseDev*)D.cases;
    if (D.rate_mode == kRatesPaper) launch_step_rates<Codec, kRatesPaper>(variant, ntiles, st, cs, tiles, S, D, parity);
    else if (D.rate_mode == kRatesPaperRaw)
        launch_step_rates<Codec, kRatesPaperRaw>(variant, ntiles, st, cs, tiles, S, D, parity);
    else launch_step_rates<Codec, kRatesGeneral>(variant, ntiles, st, cs, tiles, S, D, parity);
    return cudaGetLastError();
}

template <class Codec>
cudaError_t launch_fields_t(const DeviceState& D, int parity, const TileDev* tiles, int ntiles, double* out,
                            cudaStream_t st) {
    if (ntiles <= 0) return cudaSuccess;
    StateDev<Codec> S = make_state<Codec>(D, parity);
    fields_kernel<Codec><<<ntiles, dim3(kTR, 8), 0, st>>>((const CaseDev*)D.cases, tiles, S, out);
    return cudaGetLastError();
}

template <class Codec>
cudaError_t launch_init_t(const DeviceState& D, int parity, const TileDev* tiles8, int ntiles, const double* phi0,
                          int64_t base, cudaStream_t st) {
    if (ntiles <= 0) return cudaSuccess;
    StateDev<Codec> S = make_state<Codec>(D, parity);
    init_kernel<Codec><<<ntiles, dim3(kTR, 8), 0, st>>>((const CaseDev*)D.cases, tiles8, phi0, base, S);
    return cudaGetLastError();
}

template <class Codec>
cudaError_t launch_get_state_t(const DeviceState& D, int parity, const CaseDev& C, double* f, double* g, double* aux,
                               cudaStream_t st) {
    StateDev<Codec> S = make_state<Codec>(D, parity);
    dim3 grid((C.nr + 127) / 128, C.nz);
    get_state_kernel<Codec><<<grid, 128, 0, st>>>(C, S, f, g, aux);
    return cudaGetLastError();
}

template <class Codec>
cudaError_t launch_set_state_t(const DeviceState& D, int parity, const CaseDev& C, const double* f, const double* g,
                               const double* aux, cudaStream_t st) {
    StateDev<Codec> S = make_state<Codec>(D, parity);
    dim3 grid((C.nr + 127) / 128, C.nz);
    set_state_kernel<Codec><<<grid, 128, 0, st>>>(C, S, f, g, aux);
    return cudaGetLastError();
}

}  // namespace axilbm

#define AXILBM_INSTANTIATE(NAME, CODEC)                                                                          \
    namespace axilbm {                                                                                           \
    cudaError_t launch_step_##NAME(const DeviceState& D, int parity, int variant, const TileDev* tiles,          \
                                   int ntiles, cudaStream_t st) {                                                \
        return launch_step_t<CODEC>(D, parity, variant, tiles, ntiles, st);                                      \
    }                                                                                                            \
    cudaError_t launch_fields_##NAME(const DeviceState& D, int parity, const TileDev* tiles, int ntiles,         \
                                     double* out, cudaStream_t st) {                                             \
        return launch_fields_t<CODEC>(D, parity, tiles, ntiles, out, st);                                        \
    }                                                                                                            \
    cudaError_t launch_init_##NAME(const DeviceState& D, int parity, const TileDev* tiles8, int ntiles,          \
                                   const double* phi0, int64_t base, cudaStream_t st) {                          \
        return launch_init_t<CODEC>(D, parity, tiles8, ntiles, phi0, base, st);                                  \
    }                                                                                                            \
    cudaError_t launch_get_state_##NAME(const DeviceState& D, int parity, const CaseDev& C, double* f,           \
                                        double* g, double* aux, cudaStream_t st) {                               \
        return launch_get_state_t<CODEC>(D, parity, C, f, g, aux, st);                                           \
    }                                                                                                            \
    cudaError_t launch_set_state_##NAME(const DeviceState& D, int parity, const CaseDev& C, const double* f,     \
                                        const double* g, const double* aux, cudaStream_t st) {                   \
        return launch_set_state_t<CODEC>(D, parity, C, f, g, aux, st);                                           \
    }                                                                                                            \
    }
