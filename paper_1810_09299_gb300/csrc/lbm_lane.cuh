// lbm_lane.cuh -- the macroscopic step and both collisions of the FP16
// storage path, written once over a lane type V: one node (float) or the two
// nodes of a column that one thread updates together (float2, in the packed
// FP32x2 instructions of sm_100-family GPUs; lane x the upper node, lane y
// the lower one).  Every operation is an explicit IEEE round-to-nearest add,
// multiply or fused multiply-add, so the compiler contracts nothing on its
// own and each lane of a float2 computes exactly what the float version
// computes: every launch shape of an FP16 handle gives the same numbers.
// Quantities shared by both nodes of a column (r, 1/r, case parameters) stay
// scalars and are broadcast with bc().  The FP64, FP32 and bfloat16 paths use
// the plain forms of lbm_device.cuh.
#pragma once

#include "lbm_device.cuh"

namespace axilbm {
namespace lane {

template <class V>
struct LaneOf;
template <>
struct LaneOf<float> {
    using S = float;
};
template <>
struct LaneOf<float2> {
    using S = float;
};
template <>
struct LaneOf<double> {
    using S = double;
};

__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float vneg(float a) { return -a; }
__device__ __forceinline__ double vadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double vsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double vmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double vfma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ double vneg(double a) { return -a; }
// a - b as the exact FMA b * -1 + a (one rounding, as in IEEE subtraction)
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 vneg(float2 a) { return make_float2(-a.x, -a.y); }

template <class V>
__device__ __forceinline__ V bc(typename LaneOf<V>::S s);
template <>
__device__ __forceinline__ float bc<float>(float s) { return s; }
template <>
__device__ __forceinline__ double bc<double>(double s) { return s; }
template <>
__device__ __forceinline__ float2 bc<float2>(float s) { return make_float2(s, s); }

// FP32 reciprocal, division, square root and select of the float forms, lane
// by lane for float2.
using axilbm::rcp_;
using axilbm::div_;
using axilbm::sqrt_;
__device__ __forceinline__ float2 rcp_(float2 x) { return make_float2(rcp_(x.x), rcp_(x.y)); }
__device__ __forceinline__ float2 div_(float2 a, float2 b) { return make_float2(div_(a.x, b.x), div_(a.y, b.y)); }
__device__ __forceinline__ float2 sqrt_(float2 x) { return make_float2(sqrt_(x.x), sqrt_(x.y)); }
// t >= 0 ? a : b, lane by lane
__device__ __forceinline__ float sel_ge0(float t, float a, float b) { return t >= 0.0f ? a : b; }
__device__ __forceinline__ float2 sel_ge0(float2 t, float2 a, float2 b) {
    return make_float2(t.x >= 0.0f ? a.x : b.x, t.y >= 0.0f ? a.y : b.y);
}

// ---------------------------------------------------------------- macroscopic part
template <typename V>
struct Macro {
    using S = typename LaneOf<V>::S;
    S r, inv_r;  // of the column
    V phi, rho, nu, tau_g;
    V gz, gr, lap;
    V uz, ur, p, pstar;
    V Fz, Fr;
    V nzn, nrn, lam;
    V sg[9];
    V mg[9];  // M g (hydrodynamic moments before collision)
};

// Stencils (Eq. 39, Eq. 40) from the shared phi window centred on (a, b).
// With x1, x2 the values one and two links along c_i, d_i = 8 x1 - x2 and
// u_i = 16 x1 - x2 = 8 x1 + d_i:
//   grad phi = sum_i w_i c_i d_i / (6 cs^2),
//   lap phi  = (sum_i w_i u_i - 15 phi sum_i w_i) / (6 cs^2),
// with 6 cs^2 = 2 and sum_{i>0} w_i = 5/9, the sums grouped by weight class.
template <typename V, int LD>
__device__ __forceinline__ void stencil(const V* sphi, int a, int b, V& gz, V& gr, V& lap) {
    using S = typename LaneOf<V>::S;
    const V c0 = sphi[a * LD + b];
    V d[9], u[9];
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const V x1 = sphi[(a + cz_of(i)) * LD + (b + cr_of(i))];
        const V x2 = sphi[(a + 2 * cz_of(i)) * LD + (b + 2 * cr_of(i))];
        d[i] = vfma(bc<V>((S)8), x1, vneg(x2));
        u[i] = vfma(bc<V>((S)8), x1, d[i]);
    }
    const V h1 = bc<V>((S)(1.0 / 18.0)), h2 = bc<V>((S)(1.0 / 72.0));  // w_i / 2 on the axes and diagonals
    gz = vfma(h1, vsub(d[1], d[3]), vmul(h2, vsub(vadd(d[5], d[8]), vadd(d[6], d[7]))));
    gr = vfma(h1, vsub(d[2], d[4]), vmul(h2, vsub(vadd(d[5], d[6]), vadd(d[7], d[8]))));
    lap = vfma(h1, vadd(vadd(u[1], u[2]), vadd(u[3], u[4])),
               vfma(h2, vadd(vadd(u[5], u[6]), vadd(u[7], u[8])), vmul(bc<V>((S)(-25.0 / 6.0)), c0)));
}

// ---------------------------------------------------------------- raw moments
// The non-orthogonal basis of the raw-moment collision (the extension named
// in Sec. 4): k_0..8 = sums of x_i times 1, c_z, c_r, c_z^2 + c_r^2,
// c_z^2 - c_r^2, c_z c_r, c_z^2 c_r, c_z c_r^2, c_z^2 c_r^2.  On D2Q9 each is a
// fixed combination of the orthogonal moments of M (c^2 = (e + 4) / 3,
// c_z c_r^2 = (q_z + 2 j_z) / 3, c_z^2 c_r^2 = (eps + 2 e + 4) / 9, ...), so
// the collision stays in the orthogonal moments the step already has and maps
// the deviations into the raw basis and back.
template <typename V>
__device__ __forceinline__ void raw_from_ortho(const V* m, V* k) {
    using S = typename LaneOf<V>::S;
    const V third = bc<V>((S)(1.0 / 3.0));
    k[0] = m[0];
    k[1] = m[3];
    k[2] = m[5];
    k[3] = vmul(vfma(bc<V>((S)4), m[0], m[1]), third);
    k[4] = m[7];
    k[5] = m[8];
    k[6] = vmul(vfma(bc<V>((S)2), m[5], m[6]), third);
    k[7] = vmul(vfma(bc<V>((S)2), m[3], m[4]), third);
    k[8] = vmul(vfma(bc<V>((S)4), m[0], vfma(bc<V>((S)2), m[1], m[2])), bc<V>((S)(1.0 / 9.0)));
}
template <typename V>
__device__ __forceinline__ void ortho_from_raw(const V* k, V* m) {
    using S = typename LaneOf<V>::S;
    m[0] = k[0];
    m[3] = k[1];
    m[5] = k[2];
    m[1] = vfma(bc<V>((S)3), k[3], vmul(bc<V>((S)-4), k[0]));
    m[7] = k[4];
    m[8] = k[5];
    m[6] = vfma(bc<V>((S)3), k[6], vmul(bc<V>((S)-2), k[2]));
    m[4] = vfma(bc<V>((S)3), k[7], vmul(bc<V>((S)-2), k[1]));
    m[2] = vfma(bc<V>((S)9), k[8], vfma(bc<V>((S)-6), k[3], vmul(bc<V>((S)4), k[0])));
}
// m+ = m - A^-1 S A (m - meq) + A^-1 (I - S/2) A src, A = raw_from_ortho: the
// collision of Eq. 10 / Eq. 24 with S the rates of the raw moments.
template <typename V>
__device__ __forceinline__ void raw_relax(const V* m, const V* meq, const V* src, const V* s, V* mp) {
    using S = typename LaneOf<V>::S;
    V d[9], dk[9], sk[9], dm[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) d[i] = vsub(m[i], meq[i]);
    raw_from_ortho(d, dk);
    raw_from_ortho(src, sk);
#pragma unroll
    for (int i = 0; i < 9; ++i)
        dk[i] = vfma(vfma(bc<V>((S)-0.5), s[i], bc<V>((S)1)), sk[i], vmul(vneg(s[i]), dk[i]));
    ortho_from_raw(dk, dm);
#pragma unroll
    for (int i = 0; i < 9; ++i) mp[i] = vadd(m[i], dm[i]);
}

// Everything before the collisions for the node(s) of column j whose phi
// window is centred on (a, b), from their M g (mg) and g_0.
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
// VP (FP32 only): the first eight scalar parameters are read from the
// 16-byte aligned FP32 block of the shared case record as two 16-byte loads.
template <typename V, int LD, int RM = kRatesGeneral, bool VP = false>
__device__ __forceinline__ void node_macros(const CaseDev& C, const V* sphi, int a, int b, int j, const V* mg, V g0,
                                            V p_prev, Macro<V>& m, const typename LaneOf<V>::S* inv_r_tab = nullptr) {
    using S = typename LaneOf<V>::S;
    const CaseReal<S>& P = case_params<S>(C);
    static_assert(!VP || sizeof(S) == 4, "vector parameter loads read the FP32 block");
    float4 v0{}, v1{};
    if constexpr (VP) {
        const float4* pv = reinterpret_cast<const float4*>(&C.pf);
        v0 = pv[0];
        v1 = pv[1];
    }
    const S rho_l = VP ? (S)v0.x : P.rho_l, rho_g = VP ? (S)v0.y : P.rho_g;
    const S nu_l = VP ? (S)v0.z : P.nu_l, nu_g = VP ? (S)v0.w : P.nu_g;
    const S grav = VP ? (S)v1.x : P.grav_z, n_eps = VP ? (S)v1.y : P.n_eps;
    const S beta = VP ? (S)v1.z : P.beta, kap = VP ? (S)v1.w : P.kappa;
    const S drho = rho_l - rho_g;
    m.r = (S)j + (S)0.5;
    m.inv_r = inv_r_tab ? *inv_r_tab : rcp_(m.r);
    const S r = m.r;
    m.phi = sphi[a * LD + b];
    stencil<V, LD>(sphi, a, b, m.gz, m.gr, m.lap);
    const V phi = m.phi;
    const V pm1 = vsub(phi, bc<V>((S)1));                       // phi - 1
    m.rho = vfma(phi, bc<V>(drho), bc<V>(rho_g));               // Eq. 17
    m.nu = vfma(phi, bc<V>(nu_l - nu_g), bc<V>(nu_g));          // Eq. 35
    m.tau_g = vfma(bc<V>((S)3), m.nu, bc<V>((S)0.5));           // Eq. 34
    const V sgv = rcp_(m.tau_g);
    if constexpr (RM == kRatesPaper) {
        m.sg[1] = sgv;
    } else if constexpr (RM == kRatesPaperRaw) {
        m.sg[3] = sgv;
    } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) m.sg[i] = ((C.sg_local >> i) & 1u) ? sgv : bc<V>(P.sg[i]);
    }
    // Eq. 4 and mu~ = mu - k d_r phi / r
    const V pp1 = vmul(phi, pm1);  // phi (phi - 1)
    const V mu = vfma(bc<V>((S)4 * beta), vmul(pp1, vsub(phi, bc<V>((S)0.5))), vmul(bc<V>(-kap), m.lap));
    const V mut = vfma(bc<V>(-kap * m.inv_r), m.gr, mu);
    const V Fsz = vmul(mut, m.gz), Fsr = vmul(mut, m.gr);
    const V Gz = vmul(pm1, bc<V>(drho * grav));  // (rho - rho_l) g_z
    // interface normal and lambda (Eq. 2)
    const V ign = rcp_(vadd(sqrt_(vfma(m.gz, m.gz, vmul(m.gr, m.gr))), bc<V>(n_eps)));
    m.nzn = vmul(m.gz, ign);
    m.nrn = vmul(m.gr, ign);
    m.lam = vmul(pp1, bc<V>((S)-4 * P.inv_W));  // 4 phi (1 - phi) / W
    // hydrodynamic moments (M g, computed by the caller)
#pragma unroll
    for (int i = 0; i < 9; ++i) m.mg[i] = mg[i];
    const V Jz = m.mg[3], Jr = m.mg[5], S0 = vsub(m.mg[0], g0);
    const V dzrho = vmul(bc<V>(drho), m.gz), drrho = vmul(bc<V>(drho), m.gr);
    V sp;
    if constexpr (RM == kRatesPaper) {
        sp = vmul(bc<V>((S)0.5), m.tau_g);
    } else if constexpr (RM == kRatesPaperRaw) {
        sp = vfma(bc<V>((S)1.5), m.tau_g, bc<V>((S)-1));  // s_3 = 1/tau_g, s_8 = 1
    } else if (C.collision == 1) {
        // raw moments: Appendix C in that basis (x_0 = k_0 - k_3 + k_8)
        sp = vfma(bc<V>((S)1.5), rcp_(m.sg[3]), vfma(bc<V>((S)-0.5), rcp_(m.sg[8]), bc<V>((S)-0.5)));
    } else {
        const V s1 = m.sg[1], s2 = m.sg[2];
        sp = div_(vsub(vadd(s1, s2), vmul(s1, s2)), vmul(bc<V>((S)2), vmul(s1, s2)));
    }
    const V rho = m.rho;
    const V Fz0 = vadd(Fsz, Gz);
    m.uz = div_(vfma(bc<V>((S)0.5 * r), Fz0, Jz), vmul(bc<V>(r), rho));  // Eq. 32 (z)
    const V iDr = rcp_(vmul(rho, vfma(m.nu, bc<V>(m.inv_r), bc<V>(r))));  // 1 / (r rho + nu rho / r)
    const V uz = m.uz;
    if (C.p_coupling == 1) {
        m.pstar = p_prev;
        m.ur = vmul(vfma(bc<V>((S)0.5 * r), Fsr, vfma(bc<V>((S)0.5), m.pstar, Jr)), iDr);  // Eq. 32 (r)
        const V u2 = vfma(uz, uz, vmul(m.ur, m.ur));
        // Eq. 33
        V t = vmul(S0, bc<V>(m.inv_r));
        t = vfma(bc<V>((S)0.5), vfma(uz, dzrho, vmul(m.ur, drrho)), t);
        t = vfma(vmul(bc<V>((S)(-2.0 / 3.0)), rho), u2, t);
        t = vfma(vmul(vmul(bc<V>((S)(-4.0 / 9.0) * m.inv_r), sp), rho), m.ur, t);
        m.p = vmul(bc<V>((S)0.6), t);
    } else {
        // Eq. 32 (r) and Eq. 33 together: u_r = a + b p, p = A0 + A1 u_r - A2 u_r^2
        const V ca = vmul(vfma(bc<V>((S)0.5 * r), Fsr, Jr), iDr);
        const V cb = vmul(bc<V>((S)0.5), iDr);
        V a0 = vmul(S0, bc<V>(m.inv_r));
        a0 = vfma(vmul(bc<V>((S)0.5), uz), dzrho, a0);
        a0 = vfma(vmul(vmul(bc<V>((S)(-2.0 / 3.0)), rho), uz), uz, a0);
        const V A0 = vmul(bc<V>((S)0.6), a0);
        const V A1 = vmul(bc<V>((S)0.6), vfma(vmul(bc<V>((S)(-4.0 / 9.0) * m.inv_r), sp), rho,
                                              vmul(bc<V>((S)0.5), drrho)));
        const V A2 = vmul(bc<V>((S)0.4), rho);
        const V A2cb = vmul(A2, cb);
        const V qa = vmul(A2cb, cb);
        const V qb = vfma(vmul(bc<V>((S)2), A2cb), ca, vfma(vneg(A1), cb, bc<V>((S)1)));
        const V qc = vneg(vfma(vneg(vmul(A2, ca)), ca, vfma(A1, ca, A0)));
        const V disc = vfma(qb, qb, vmul(vmul(bc<V>((S)-4), qa), qc));
        // both roots' divisions, then the select (selecting the numerator and
        // denominator first is bit-identical and measured 2 % slower in the
        // packed two-node step)
        m.p = sel_ge0(disc, div_(vmul(bc<V>((S)-2), qc), vadd(qb, sqrt_(disc))), div_(vneg(qc), qb));
        m.pstar = m.p;
        m.ur = vfma(cb, m.p, ca);
    }
    // Eq. 30
    m.Fz = vmul(bc<V>(r), Fz0);
    m.Fr = vfma(bc<V>(r), Fsr, vfma(vmul(vmul(bc<V>((S)-2 * m.inv_r), rho), m.nu), m.ur, m.pstar));
}

// ---------------------------------------------------------------- collisions
// Phase field (Eq. 19 in moment space with Eq. 21-23).  chi = (r phi u_z,
// r phi u_r + M phi); the time derivative of Eq. 38 uses chi^{n-1}.
template <typename V, int RM = kRatesGeneral>
__device__ __forceinline__ void collide_f(const CaseDev& C, const Macro<V>& m, const V* mf, V chi_z_prev,
                                          V chi_r_prev, V& chi_z, V& chi_r, V* mp) {
    using S = typename LaneOf<V>::S;
    const CaseReal<S>& P = case_params<S>(C);
    const V rphi = mf[0];  // = r phi exactly (phi is sum f / r)
    const V rp = vmul(bc<V>(m.r), m.phi);
    chi_z = vmul(rp, m.uz);
    chi_r = vfma(rp, m.ur, vmul(bc<V>(P.mob), m.phi));
    const V rl3 = vmul(bc<V>(m.r * (S)(1.0 / 3.0)), m.lam);
    const V mR1 = vfma(rl3, m.nzn, vsub(chi_z, chi_z_prev));
    const V mR2 = vfma(rl3, m.nrn, vsub(chi_r, chi_r_prev));
    const V zero = bc<V>((S)0);
    const V meq[9] = {rphi, vmul(bc<V>((S)-2), rphi), rphi, chi_z, vneg(chi_z), chi_r, vneg(chi_r), zero, zero};
    const V mR[9] = {zero, zero, zero, mR1, vneg(mR1), mR2, vneg(mR2), zero, zero};
    if constexpr (RM != kRatesGeneral) {
        // unit rates: m0 is conserved, m1, m2, m7, m8 take their equilibria.
        // The raw-moment pattern (rate s on c_z, c_r, c_z^2 c_r, c_z c_r^2)
        // spans the same rate subspaces, so it is this very operator; its s
        // is the rate of raw moment 1.
        const S s = RM == kRatesPaperRaw ? P.sf[1] : P.sf[3], h = (S)1 - (S)0.5 * s;
        mp[0] = rphi;
        mp[1] = meq[1];
        mp[2] = meq[2];
#pragma unroll
        for (int k = 3; k < 7; ++k) mp[k] = vfma(bc<V>(h), mR[k], vfma(bc<V>(-s), vsub(mf[k], meq[k]), mf[k]));
        mp[7] = zero;
        mp[8] = zero;
    } else if (C.collision == 1) {
        V s[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) s[k] = bc<V>(P.sf[k]);
        raw_relax<V>(mf, meq, mR, s, mp);
    } else {
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const S s = P.sf[k];
            mp[k] = vfma(bc<V>((S)1 - (S)0.5 * s), mR[k], vfma(bc<V>(-s), vsub(mf[k], meq[k]), mf[k]));
        }
    }
}

// Hydrodynamics (Eq. 24 in moment space with Eq. 36-37).
template <typename V, int RM = kRatesGeneral>
__device__ __forceinline__ void collide_g(const CaseDev& C, const Macro<V>& m, V* mp) {
    using S = typename LaneOf<V>::S;
    const CaseReal<S>& P = case_params<S>(C);
    const S r = m.r;
    const V rho = m.rho, uz = m.uz, ur = m.ur, p = m.p;
    const V uzz = vmul(uz, uz), urr = vmul(ur, ur);
    const V u2 = vadd(uzz, urr);
    const S rdrho = r * (P.rho_l - P.rho_g);
    const V dz_rr = vmul(bc<V>(rdrho), m.gz);          // d_z (r rho)
    const V dr_rr = vfma(bc<V>(rdrho), m.gr, rho);     // d_r (r rho)
    const V udr = vfma(uz, dz_rr, vmul(ur, dr_rr));
    const V rr = vmul(bc<V>(r), rho);
    const V rho_ur = vmul(rho, ur);
    const V rrz = vmul(rr, uz), rrr = vmul(rr, ur);
    const V meq[9] = {bc<V>((S)0),
                      vmul(bc<V>((S)3 * r), vfma(rho, u2, vmul(bc<V>((S)2), p))),
                      vmul(bc<V>((S)-3 * r), vfma(rho, u2, vmul(bc<V>((S)3), p))),
                      rrz, vneg(rrz), rrr, vneg(rrr),
                      vmul(rr, vsub(uzz, urr)),
                      vmul(rrr, uz)};
    const V MT[9] = {vsub(udr, rho_ur),  // = r u . grad rho
                     vmul(bc<V>((S)2), rho_ur),
                     vsub(vneg(udr), rho_ur),
                     m.Fz, vneg(m.Fz), m.Fr, vneg(m.Fr),
                     vmul(bc<V>((S)(2.0 / 3.0)), vfma(uz, dz_rr, vneg(vmul(ur, dr_rr)))),
                     vmul(bc<V>((S)(1.0 / 3.0)), vfma(uz, dr_rr, vmul(ur, dz_rr)))};
    if constexpr (RM == kRatesPaper) {
        const V s = m.sg[1], h = vfma(bc<V>((S)-0.5), s, bc<V>((S)1));
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            if (k == 1 || k == 7 || k == 8) mp[k] = vfma(h, MT[k], vfma(vneg(s), vsub(m.mg[k], meq[k]), m.mg[k]));
            else mp[k] = vfma(bc<V>((S)0.5), MT[k], meq[k]);
        }
    } else if constexpr (RM == kRatesPaperRaw) {
        // raw moments: the three second moments at 1/tau_g, the rest at 1
        const V s = m.sg[3], one = bc<V>((S)1);
        const V rates[9] = {one, one, one, s, s, s, one, one, one};
        raw_relax<V>(m.mg, meq, MT, rates, mp);
    } else if (C.collision == 1) {
        raw_relax<V>(m.mg, meq, MT, m.sg, mp);
    } else {
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const V s = m.sg[k];
            mp[k] = vfma(vfma(bc<V>((S)-0.5), s, bc<V>((S)1)), MT[k], vfma(vneg(s), vsub(m.mg[k], meq[k]), m.mg[k]));
        }
    }
}


}  // namespace lane
}  // namespace axilbm
