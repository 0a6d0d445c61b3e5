// Device code shared by the plain and the batched force kernels: the Ewald
// rational approximations, the pair interaction and the per-work-item loop of
// the cluster pair algorithm (paper Sec. V.A).
#pragma once
#include "ewald_rational.h"
#include "nb_internal.cuh"

namespace nbk {

static_assert(NB_EW_ZMAX == (float)NB_EW_ZMAX_D, "Ewald fit range");


// Hardware approximations in their flush-to-zero forms.  Without .ftz the
// compiler wraps each one in a rescaling for denormal inputs (a compare, two
// multiplies and a select); no input here is denormal (squared distances are
// clamped to at most rc^2 and at least the closest pair's, denominators of the
// rationals are >= 1), so the results are the same and the wrapper is dead code
// that cost 9% of the force kernel's instructions.
__device__ __forceinline__ float rsq_approx(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// 2^x (the hardware approximation, flush-to-zero form)
__device__ __forceinline__ float ex2_approx(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float div_approx(float a, float b) {
    float r;
    asm("div.approx.ftz.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}


__device__ __forceinline__ float ew_h(float s) {
    float p = fmaf(NB_EW_HP6, s, NB_EW_HP5);
    p = fmaf(p, s, NB_EW_HP4);
    p = fmaf(p, s, NB_EW_HP3);
    p = fmaf(p, s, NB_EW_HP2);
    p = fmaf(p, s, NB_EW_HP1);
    p = fmaf(p, s, NB_EW_HP0);
    float q = fmaf(NB_EW_HQ5, s, NB_EW_HQ4);
    q = fmaf(q, s, NB_EW_HQ3);
    q = fmaf(q, s, NB_EW_HQ2);
    q = fmaf(q, s, NB_EW_HQ1);
    q = fmaf(q, s, 1.0f);
    return div_approx(p, q);
}

// exp(-x) for 0 <= x < 80: x = n ln2 + u (Cody-Waite reduction; n * LN2_HI is
// exact), exp(-u) by the degree-7 polynomial 1 + w q(w) with w = -u, times 2^-n
//
// n = rint(x log2 e) by the 1.5 * 2^23 shift in one FMA: m = x log2 e + 1.5 * 2^23,
// rounded once, is an integer whose low mantissa bits hold n (0 <= n < 2^22; ties go
// to even, so n is the round-half-even integer nearest the exact product), -n =
// 1.5 * 2^23 - m is exact, and the scale 2^-n has the bits 0x3f800000 - (bits(m) << 23).
// No float -> int conversions.
__device__ __forceinline__ float ew_expm(float x) {
    const float m = __fmaf_rn(x, NB_EXP_LOG2E, 12582912.0f);
    const float nn = __fsub_rn(12582912.0f, m);
    float u = fmaf(nn, NB_EXP_LN2_HI, x);
    u = fmaf(nn, NB_EXP_LN2_LO, u);
    const float w = -u;
    float q = fmaf(NB_EXP_C7, w, NB_EXP_C6);
    q = fmaf(q, w, NB_EXP_C5);
    q = fmaf(q, w, NB_EXP_C4);
    q = fmaf(q, w, NB_EXP_C3);
    q = fmaf(q, w, NB_EXP_C2);
    q = fmaf(q, w, NB_EXP_C1);
    const float p = fmaf(q, w, 1.0f);
    return p * __int_as_float(0x3f800000 - (__float_as_int(m) << 23));
}

// Reciprocal of q > 0 within about half an ulp: the hardware approximation
// refined by one Newton step on the FMA residual.  The energy kernels divide by
// it in X(z); the bare approximation (a fast division) carries a rounding bias
// that varies with z, and the Coulomb energy of water -- a sum whose terms cancel
// about 3000-fold -- turned that into a relative energy error of 2e-6.
__device__ __forceinline__ float rcp_refined(float q) {
    const float r = rcp_approx(q);
    return fmaf(r, fmaf(-q, r, 1.0f), r);
}

// X(z) = exp(z^2) erfc(z), a (6,6) rational in t = z / ZMAX (the argument)
__device__ __forceinline__ float ew_x(float t) {
    float p = fmaf(NB_EW_XP6, t, NB_EW_XP5);
    p = fmaf(p, t, NB_EW_XP4);
    p = fmaf(p, t, NB_EW_XP3);
    p = fmaf(p, t, NB_EW_XP2);
    p = fmaf(p, t, NB_EW_XP1);
    p = fmaf(p, t, NB_EW_XP0);
    float q = fmaf(NB_EW_XQ6, t, NB_EW_XQ5);
    q = fmaf(q, t, NB_EW_XQ4);
    q = fmaf(q, t, NB_EW_XQ3);
    q = fmaf(q, t, NB_EW_XQ2);
    q = fmaf(q, t, NB_EW_XQ1);
    q = fmaf(q, t, 1.0f);
    return p * rcp_refined(q);
}

// Packed FP32 (sm_100 and later): one FFMA2 / FMUL2 / FADD2 instruction performs
// the operation on both components of a float2, each rounded exactly as the
// scalar operation.  The force kernel evaluates two pairs per lane, so their
// arithmetic runs on pairs of values and takes half the issue slots.
__device__ __forceinline__ float2 p2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 pneg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 psub(float2 a, float2 b) { return __fadd2_rn(a, pneg(b)); }

// ew_h, ew_expm and ew_x on two values (the same operations per component)
__device__ __forceinline__ float2 ew_h2(float2 s) {
    float2 p = pfma(p2(NB_EW_HP6), s, p2(NB_EW_HP5));
    p = pfma(p, s, p2(NB_EW_HP4));
    p = pfma(p, s, p2(NB_EW_HP3));
    p = pfma(p, s, p2(NB_EW_HP2));
    p = pfma(p, s, p2(NB_EW_HP1));
    p = pfma(p, s, p2(NB_EW_HP0));
    float2 q = pfma(p2(NB_EW_HQ5), s, p2(NB_EW_HQ4));
    q = pfma(q, s, p2(NB_EW_HQ3));
    q = pfma(q, s, p2(NB_EW_HQ2));
    q = pfma(q, s, p2(NB_EW_HQ1));
    q = pfma(q, s, p2(1.0f));
    return make_float2(div_approx(p.x, q.x), div_approx(p.y, q.y));
}

__device__ __forceinline__ float2 ew_expm2(float2 x) {
    const float2 m = pfma(x, p2(NB_EXP_LOG2E), p2(12582912.0f));
    const float2 nn = psub(p2(12582912.0f), m);  // -n, exact
    float2 u = pfma(nn, p2(NB_EXP_LN2_HI), x);
    u = pfma(nn, p2(NB_EXP_LN2_LO), u);
    const float2 w = pneg(u);
    float2 q = pfma(p2(NB_EXP_C7), w, p2(NB_EXP_C6));
    q = pfma(q, w, p2(NB_EXP_C5));
    q = pfma(q, w, p2(NB_EXP_C4));
    q = pfma(q, w, p2(NB_EXP_C3));
    q = pfma(q, w, p2(NB_EXP_C2));
    q = pfma(q, w, p2(NB_EXP_C1));
    const float2 p = pfma(q, w, p2(1.0f));
    return pmul(p, make_float2(__int_as_float(0x3f800000 - (__float_as_int(m.x) << 23)),
                               __int_as_float(0x3f800000 - (__float_as_int(m.y) << 23))));
}

__device__ __forceinline__ float2 ew_x2(float2 t) {
    float2 p = pfma(p2(NB_EW_XP6), t, p2(NB_EW_XP5));
    p = pfma(p, t, p2(NB_EW_XP4));
    p = pfma(p, t, p2(NB_EW_XP3));
    p = pfma(p, t, p2(NB_EW_XP2));
    p = pfma(p, t, p2(NB_EW_XP1));
    p = pfma(p, t, p2(NB_EW_XP0));
    float2 q = pfma(p2(NB_EW_XQ6), t, p2(NB_EW_XQ5));
    q = pfma(q, t, p2(NB_EW_XQ4));
    q = pfma(q, t, p2(NB_EW_XQ3));
    q = pfma(q, t, p2(NB_EW_XQ2));
    q = pfma(q, t, p2(NB_EW_XQ1));
    q = pfma(q, t, p2(1.0f));
    float2 r = make_float2(rcp_approx(q.x), rcp_approx(q.y));  // rcp_refined per component
    r = pfma(r, pfma(pneg(q), r, p2(1.0f)), r);
    return pmul(p, r);
}

// Periodic shift of a work item split between the two sides of each pair so
// that every shifted coordinate stays exact.  For shift s (per axis) the pair
// vector is x_i - x_j + s L.  On an axis with s = -1 the i-atoms lie near the
// upper face and x_i - L is exact (Sterbenz); with s = +1 the j-atoms lie near
// the upper face and x_j - L is exact.  Adding L to a coordinate near 0
// instead would round away the low bits of L and bias every such pair alike.
// L = Lhi + Llo (float pair); the Llo parts are added after the exact step.
struct ShiftSplit {
    float ihi[3], ilo[3];  // x_i' = (x_i + ihi) + ilo
    float jhi[3], jlo[3];  // x_j' = (x_j - jhi) - jlo
    bool jshift;
};

__device__ __forceinline__ ShiftSplit make_shift(int sidx, const float *Lhi, const float *Llo) {
    ShiftSplit r;
    int s[3];
    shift_of(sidx, s[0], s[1], s[2]);
    r.jshift = false;
    for (int k = 0; k < 3; k++) {
        r.ihi[k] = s[k] < 0 ? -Lhi[k] : 0.f;
        r.ilo[k] = s[k] < 0 ? -Llo[k] : 0.f;
        r.jhi[k] = s[k] > 0 ? Lhi[k] : 0.f;
        r.jlo[k] = s[k] > 0 ? Llo[k] : 0.f;
        r.jshift |= s[k] > 0;
    }
    return r;
}

__device__ __forceinline__ float4 shift_i(float4 p, const ShiftSplit &sh) {
    p.x = (p.x + sh.ihi[0]) + sh.ilo[0];
    p.y = (p.y + sh.ihi[1]) + sh.ilo[1];
    p.z = (p.z + sh.ihi[2]) + sh.ilo[2];
    return p;
}

__device__ __forceinline__ float4 shift_j(float4 p, const ShiftSplit &sh) {
    p.x = (p.x - sh.jhi[0]) - sh.jlo[0];
    p.y = (p.y - sh.jhi[1]) - sh.jlo[1];
    p.z = (p.z - sh.jhi[2]) - sh.jlo[2];
    return p;
}

// Compensated (Kahan) accumulation of the per-entry energy subtotals: the
// energy totals of small systems are sums of many terms that nearly cancel, so
// the running-sum rounding of a plain FP32 accumulator would dominate.
struct KSum {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    // merge another compensated sum (error-free two-sum of the leading parts)
    __device__ __forceinline__ void merge(float s2, float c2) {
        const float t = s + s2;
        const float bp = t - s;
        const float err = (s - (t - bp)) + (s2 - bp);
        s = t;
        c = c + c2 - err;
    }
};

// One pair: returns the scalar force phi (force on i = phi * d), adds energies.
// Force-only kernels get qi pre-multiplied by the Coulomb constant f; energy
// kernels get the raw charge and apply f to the force here and to the energy
// once, in FP64, after the reduction (a rounded f would bias every pair alike).
template <int COUL, bool EN>
__device__ __forceinline__ float pair_phi(const SysView &v, const float2 *__restrict__ ljt,
                                          const float4 *__restrict__ lje, float3 d, float qi, float qj, int tpair,
                                          bool bit, float &elj, float &ec) {
    float r2 = fmaf(d.z, d.z, fmaf(d.y, d.y, d.x * d.x));
    const bool in = bit && (r2 < v.rc2);
    r2 = in ? r2 : v.rc2;
    float rinv = rsq_approx(r2);
    if (EN) rinv = rsqrt_refine(r2, rinv);
    const float rinv2 = rinv * rinv;
    const float rinv6 = rinv2 * rinv2 * rinv2;
    const float2 lj = ljt[tpair];  // (6 C6, 12 C12)
    const float flj = rinv6 * fmaf(lj.y, rinv6, -lj.x);
    const float qq = qi * qj;
    float fc = 0.f, erfcz = 0.f;
    if (COUL == NB_COULOMB_RF) {
        fc = qq * fmaf(rinv, rinv2, -2.0f * v.k_rf);
    } else if (COUL == NB_COULOMB_EWALD) {
        if (EN) {
            // one exp(-z^2) serves the energy, erfc(z) = exp(-z^2) X(z), and the force;
            // t = z / ZMAX = (beta / ZMAX) r and z^2 = beta^2 r^2 take beta / ZMAX and
            // beta^2 as float pairs, so their FP32 rounding leaves no error that grows
            // with z (each pair of the energy sum then carries only unbiased roundings;
            // ZMAX is a power of two, so t is z / ZMAX exactly)
            const float r = r2 * rinv;
            const float ex = ew_expm(fmaf(r2, v.ew_beta2, r2 * v.ew_beta2_lo));
            erfcz = ex * ew_x(fmaf(v.ew_bt, r, v.ew_bt_lo * r));
            fc = qq * rinv2 * fmaf(erfcz, rinv, v.ew_2bsp * ex);
        } else {
            fc = qq * fmaf(rinv, rinv2, -v.ew_beta3 * ew_h(r2 * v.ew_s));
        }
    }
    if (EN) fc *= v.coul_f;
    float phi = fmaf(flj, rinv2, fc);
    phi = in ? phi : 0.f;
    if (EN) {
        const float4 le = lje[tpair];  // (C6, C12, C12/rc^12 - C6/rc^6, -)
        const float vlj = fmaf(rinv6, fmaf(le.y, rinv6, -le.x), -le.z);
        float vc = 0.f;
        if (COUL == NB_COULOMB_RF) {
            // 1/r as a float pair (rinv + rlo) from the exact residual 1 - r2 rinv^2;
            // (rinv - c_rf) is then exact near the cut-off, where the terms cancel
            const float t_hi = rinv * rinv;
            const float t_lo = fmaf(rinv, rinv, -t_hi);
            const float e = fmaf(-r2, t_hi, 1.0f) - r2 * t_lo;
            const float rlo = 0.5f * rinv * e;
            vc = (rinv - v.c_rf) + (fmaf(v.k_rf, r2, -v.c_rf_lo) + rlo);
        } else if (COUL == NB_COULOMB_EWALD) {
            vc = fmaf(erfcz, rinv, -v.ew_shift);
        }
        elj += in ? vlj : 0.f;
        ec += in ? qq * vc : 0.f;
    }
    return phi;
}

// Lennard-Jones parameters of the two pairs of a packed iteration, one component
// per pair: 6 C6, 12 C12 (forces) and C6, C12, C12/rc^12 - C6/rc^6 (energies).
struct Lj2 {
    float2 f6, f12, e6, e12, sh;
};

// The type-pair tables (T x T) and, for few types, the same values rearranged by
// (i-type, j-type of the lower j-atom, j-type of the upper j-atom), T^3 entries, so
// that one load yields both pairs' parameters already packed.
struct LjTables {
    const float2 *lj;   // [T*T] (6 C6, 12 C12)
    const float4 *lje;  // [T*T] (C6, C12, C12/rc^12 - C6/rc^6, 0)
    const float4 *l3f;  // [T^3] (6 C6, 6 C6', 12 C12, 12 C12')
    const float4 *l3e;  // [T^3] (C6, C6', C12, C12')
    const float2 *l3s;  // [T^3] (shift, shift')
};

template <bool EN>
__device__ __forceinline__ Lj2 lj_gather(const LjTables &t, int tp0, int tp1) {
    Lj2 r;
    const float2 la = t.lj[tp0], lb = t.lj[tp1];
    r.f6 = make_float2(la.x, lb.x);
    r.f12 = make_float2(la.y, lb.y);
    if (EN) {
        const float4 ea = t.lje[tp0], eb = t.lje[tp1];
        r.e6 = make_float2(ea.x, eb.x);
        r.e12 = make_float2(ea.y, eb.y);
        r.sh = make_float2(ea.z, eb.z);
    }
    return r;
}

template <bool EN>
__device__ __forceinline__ Lj2 lj_triple(const LjTables &t, int idx) {
    Lj2 r;
    const float4 f = t.l3f[idx];
    r.f6 = make_float2(f.x, f.y);
    r.f12 = make_float2(f.z, f.w);
    if (EN) {
        const float4 e = t.l3e[idx];
        r.e6 = make_float2(e.x, e.y);
        r.e12 = make_float2(e.z, e.w);
        r.sh = t.l3s[idx];
    }
    return r;
}

// Two pairs at once: pair_phi's operations, in the same order, on float2 values
// (component 0: the first pair, component 1: the second; i-charges qi and
// j-charges qj per component).  Energies are added per component to elj / ec.
template <int COUL, bool EN>
__device__ __forceinline__ float2 pair_phi2(const SysView &v, const Lj2 &lj, float2 dx, float2 dy, float2 dz, float2 qi,
                                            float2 qj, bool b0, bool b1, float2 &elj, float2 &ec) {
    float2 r2 = pfma(dz, dz, pfma(dy, dy, pmul(dx, dx)));
    const bool in0 = b0 && (r2.x < v.rc2), in1 = b1 && (r2.y < v.rc2);
    r2.x = in0 ? r2.x : v.rc2;
    r2.y = in1 ? r2.y : v.rc2;
    float2 rinv = make_float2(rsq_approx(r2.x), rsq_approx(r2.y));
    if (EN) {  // rsqrt_refine
        const float2 e = pfma(pneg(pmul(r2, rinv)), rinv, p2(1.0f));
        rinv = pfma(pmul(p2(0.5f), rinv), e, rinv);
    }
    const float2 rinv2 = pmul(rinv, rinv);
    const float2 rinv6 = pmul(pmul(rinv2, rinv2), rinv2);
    const float2 flj = pmul(rinv6, pfma(lj.f12, rinv6, pneg(lj.f6)));
    const float2 qq = pmul(qi, qj);
    float2 fc = p2(0.f), erfcz = p2(0.f);
    if (COUL == NB_COULOMB_RF) {
        fc = pmul(qq, pfma(rinv, rinv2, p2(-2.0f * v.k_rf)));
    } else if (COUL == NB_COULOMB_EWALD) {
        if (EN) {
            const float2 r = pmul(r2, rinv);
            const float2 ex = ew_expm2(pfma(r2, p2(v.ew_beta2), pmul(r2, p2(v.ew_beta2_lo))));
            erfcz = pmul(ex, ew_x2(pfma(p2(v.ew_bt), r, pmul(p2(v.ew_bt_lo), r))));
            fc = pmul(pmul(qq, rinv2), pfma(erfcz, rinv, pmul(p2(v.ew_2bsp), ex)));
        } else {
            fc = pmul(qq, pfma(rinv, rinv2, pmul(p2(-v.ew_beta3), ew_h2(pmul(r2, p2(v.ew_s))))));
        }
    }
    if (EN) fc = pmul(fc, p2(v.coul_f));
    float2 phi = pfma(flj, rinv2, fc);
    phi.x = in0 ? phi.x : 0.f;
    phi.y = in1 ? phi.y : 0.f;
    if (EN) {
        float2 vlj = pfma(rinv6, pfma(lj.e12, rinv6, pneg(lj.e6)), pneg(lj.sh));
        float2 vc = p2(0.f);
        if (COUL == NB_COULOMB_RF) {
            const float2 t_hi = pmul(rinv, rinv);
            const float2 t_lo = pfma(rinv, rinv, pneg(t_hi));
            const float2 e = psub(pfma(pneg(r2), t_hi, p2(1.0f)), pmul(r2, t_lo));
            const float2 rlo = pmul(pmul(p2(0.5f), rinv), e);
            vc = padd(psub(rinv, p2(v.c_rf)), padd(pfma(p2(v.k_rf), r2, p2(-v.c_rf_lo)), rlo));
        } else if (COUL == NB_COULOMB_EWALD) {
            vc = pfma(erfcz, rinv, p2(-v.ew_shift));
        }
        float2 qv = pmul(qq, vc);
        vlj.x = in0 ? vlj.x : 0.f;
        vlj.y = in1 ? vlj.y : 0.f;
        qv.x = in0 ? qv.x : 0.f;
        qv.y = in1 ? qv.y : 0.f;
        elj = padd(elj, vlj);
        ec = padd(ec, qv);
    }
    return phi;
}

// Evaluate work item w (nj > 0 inner entries) with one warp.  s_xi / s_ti are
// this warp's 64-entry staging arrays and s_fi its i-force accumulators
// ([8 clusters][3][32 lanes] floats, conflict-free); ljt the type-pair tables
// (shared or global memory; LJ3: the i-clusters that interact with both j-halves
// read the rearranged T^3 table, one load for both pairs).  Forces are added to v.f; energies and the virial
// sum of r (x) F go to the caller's per-lane accumulators.  The i-cluster loop
// walks the set bits of the interaction mask (a warp-uniform loop) and is not
// unrolled, so the kernel stays small enough for the instruction cache and the
// i-forces of the 8 clusters live in shared memory rather than in registers.
//
// PRUNE (first use of a new list, Sec. V.D): the entries are the outer list's
// (one 8-bit mask for both j-halves); while computing the forces the warp also
// records, per i-cluster and j-half, whether any atom pair is closer than r_in,
// and writes those half masks to v.kept for the compaction into the inner list.
template <int COUL, bool EN, bool VIR, bool PRUNE = false, bool LJ3 = false>
__device__ __forceinline__ void process_item(const SysView &v, int w, int nj, const LjTables &ljt,
                                             float4 *s_xi, int *s_ti, float *s_fi, KSum &elj, KSum &ec,
                                             float (&vr)[9]) {
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu;
    const int4 it = v.items[w];
    const int si = it.x, j0 = it.z;
    const ShiftSplit sh = make_shift(it.y, v.box_hi, v.box_lo);
    for (int h = 0; h < 2; h++) {
        const int at = lane + 32 * h;
        float4 p = shift_i(v.xq[si * NB_SCA + at], sh);
        if (!EN) p.w *= v.coul_f;
        s_xi[at] = p;
        s_ti[at] = v.type[si * NB_SCA + at] * v.T;
    }
#pragma unroll
    for (int k = 0; k < 3 * NB_SCL; k++) s_fi[k * 32 + lane] = 0.f;
    __syncwarp();
    const int ti = lane & 7, tj = lane >> 3;
    float4 org = make_float4(0.f, 0.f, 0.f, 0.f);
    if (VIR) org = s_xi[0];

    for (int e = 0; e < nj; e++) {
        const int2 ent = v.cj[j0 + e];
        const int cj = PRUNE ? ent.x : inner_cj(ent), mg = entry_group(ent);
        const int lo = PRUNE ? (ent.y & 0xff) : inner_lo(ent), hi = PRUNE ? lo : inner_hi(ent);
        int keep_lo = 0, keep_hi = 0;  // PRUNE: half masks that survive r_in
        float4 xj0 = v.xq[cj * NB_CL + tj], xj1 = v.xq[cj * NB_CL + tj + 4];
        if (sh.jshift) {
            xj0 = shift_j(xj0, sh);
            xj1 = shift_j(xj1, sh);
        }
        const int tj0 = v.type[cj * NB_CL + tj], tj1 = v.type[cj * NB_CL + tj + 4];
        const int tjj = LJ3 ? tj0 * v.T + tj1 : 0;  // (j-type, j-type') row of the T^3 table
        // exclusion bits of the lane's two pairs for every i-cluster k (bits 2k, 2k + 1)
        const unsigned mw = mg ? (unsigned)v.mask_lanes[(size_t)(mg - 1) * 32 + lane] : 0xffffu;
        // the lane's two j-atoms as packed pairs (component 0: tj, component 1: tj + 4)
        const float2 jx = make_float2(xj0.x, xj1.x), jy = make_float2(xj0.y, xj1.y);
        const float2 jz = make_float2(xj0.z, xj1.z), jq = make_float2(xj0.w, xj1.w);
        float2 fjx = p2(0.f), fjy = p2(0.f), fjz = p2(0.f);  // j-forces of the two atoms
        float2 elj2 = p2(0.f), ec2 = p2(0.f);
        float elj_e = 0.f, ec_e = 0.f;
        // i-clusters that interact with both j-halves: two pairs per lane, packed
        int both = lo & hi;
#pragma unroll 1
        while (both) {
            const int k = __ffs(both) - 1;
            both &= both - 1;
            const bool b0 = (mw >> (2 * k)) & 1u, b1 = (mw >> (2 * k + 1)) & 1u;
            const int tio = s_ti[k * NB_CL + ti];
            const float4 xi = s_xi[k * NB_CL + ti];
            const float2 dx = psub(p2(xi.x), jx), dy = psub(p2(xi.y), jy), dz = psub(p2(xi.z), jz);
            const float2 qi2 = p2(xi.w);
            if (PRUNE) {  // the separate prune pass's test, r^2 - r_in^2 < 0, rounded alike
                const float2 q = pfma(dz, dz, pfma(dy, dy, pfma(dx, dx, p2(-v.rin2))));
                keep_lo |= (int)__any_sync(full, __float_as_uint(q.x) >> 31) << k;
                keep_hi |= (int)__any_sync(full, __float_as_uint(q.y) >> 31) << k;
            }
            const Lj2 lj = LJ3 ? lj_triple<EN>(ljt, tio * v.T + tjj) : lj_gather<EN>(ljt, tio + tj0, tio + tj1);
            const float2 p = pair_phi2<COUL, EN>(v, lj, dx, dy, dz, qi2, jq, b0, b1, elj2, ec2);
            // force p d on i and -p d on j.  Each product is fused into its accumulation where
            // that measured faster: the T^3-table kernels for forces alone and for forces +
            // energies + virial.  With energies or the virial alone, and in the T x T-table
            // kernels, the fused form was 3-5% slower.
            float *fk = s_fi + k * 96 + lane;
            if (LJ3 && EN == VIR) {
                fk[0] = __fmaf_rn(p.y, dx.y, __fmaf_rn(p.x, dx.x, fk[0]));
                fk[32] = __fmaf_rn(p.y, dy.y, __fmaf_rn(p.x, dy.x, fk[32]));
                fk[64] = __fmaf_rn(p.y, dz.y, __fmaf_rn(p.x, dz.x, fk[64]));
                const float2 pn = pneg(p);
                fjx = pfma(pn, dx, fjx);
                fjy = pfma(pn, dy, fjy);
                fjz = pfma(pn, dz, fjz);
            } else {
                const float2 ax = pmul(p, dx), ay = pmul(p, dy), az = pmul(p, dz);
                fk[0] += ax.x + ax.y;
                fk[32] += ay.x + ay.y;
                fk[64] += az.x + az.y;
                fjx = psub(fjx, ax);
                fjy = psub(fjy, ay);
                fjz = psub(fjz, az);
            }
        }
        // i-clusters that the prune kept for one j-half only: two such i-clusters share a
        // packed iteration (each component its own i-atom, j-atom and mask bit)
        int one = lo ^ hi;
#pragma unroll 1
        while (__popc(one) >= 2) {
            const int ka = __ffs(one) - 1;
            one &= one - 1;
            const int kb = __ffs(one) - 1;
            one &= one - 1;
            const bool ua = (hi >> ka) & 1, ub = (hi >> kb) & 1;  // warp-uniform
            const bool ba = (mw >> (2 * ka + (ua ? 1 : 0))) & 1u, bb = (mw >> (2 * kb + (ub ? 1 : 0))) & 1u;
            const float4 xia = s_xi[ka * NB_CL + ti], xib = s_xi[kb * NB_CL + ti];
            const float4 xja = ua ? xj1 : xj0, xjb = ub ? xj1 : xj0;
            const float2 dx = psub(make_float2(xia.x, xib.x), make_float2(xja.x, xjb.x));
            const float2 dy = psub(make_float2(xia.y, xib.y), make_float2(xja.y, xjb.y));
            const float2 dz = psub(make_float2(xia.z, xib.z), make_float2(xja.z, xjb.z));
            const Lj2 lj = lj_gather<EN>(ljt, s_ti[ka * NB_CL + ti] + (ua ? tj1 : tj0),
                                         s_ti[kb * NB_CL + ti] + (ub ? tj1 : tj0));
            const float2 p = pair_phi2<COUL, EN>(v, lj, dx, dy, dz, make_float2(xia.w, xib.w),
                                                 make_float2(xja.w, xjb.w), ba, bb, elj2, ec2);
            float *fa = s_fi + ka * 96 + lane;
            float *fb = s_fi + kb * 96 + lane;
            fa[0] = __fmaf_rn(p.x, dx.x, fa[0]);
            fa[32] = __fmaf_rn(p.x, dy.x, fa[32]);
            fa[64] = __fmaf_rn(p.x, dz.x, fa[64]);
            fb[0] = __fmaf_rn(p.y, dx.y, fb[0]);
            fb[32] = __fmaf_rn(p.y, dy.y, fb[32]);
            fb[64] = __fmaf_rn(p.y, dz.y, fb[64]);
            if (ua) {
                fjx.y = __fmaf_rn(-p.x, dx.x, fjx.y);
                fjy.y = __fmaf_rn(-p.x, dy.x, fjy.y);
                fjz.y = __fmaf_rn(-p.x, dz.x, fjz.y);
            } else {
                fjx.x = __fmaf_rn(-p.x, dx.x, fjx.x);
                fjy.x = __fmaf_rn(-p.x, dy.x, fjy.x);
                fjz.x = __fmaf_rn(-p.x, dz.x, fjz.x);
            }
            if (ub) {
                fjx.y = __fmaf_rn(-p.y, dx.y, fjx.y);
                fjy.y = __fmaf_rn(-p.y, dy.y, fjy.y);
                fjz.y = __fmaf_rn(-p.y, dz.y, fjz.y);
            } else {
                fjx.x = __fmaf_rn(-p.y, dx.y, fjx.x);
                fjy.x = __fmaf_rn(-p.y, dy.y, fjy.x);
                fjz.x = __fmaf_rn(-p.y, dz.y, fjz.x);
            }
        }
        if (one) {  // the last single-half i-cluster: one pair per lane
            const int k = __ffs(one) - 1;
            const bool upper = (hi >> k) & 1;  // warp-uniform
            const bool b = (mw >> (2 * k + (upper ? 1 : 0))) & 1u;
            const float4 xj = upper ? xj1 : xj0;
            const float4 xi = s_xi[k * NB_CL + ti];
            const int tio = s_ti[k * NB_CL + ti];
            const float3 d = make_float3(xi.x - xj.x, xi.y - xj.y, xi.z - xj.z);
            const float p = pair_phi<COUL, EN>(v, ljt.lj, ljt.lje, d, xi.w, xj.w, tio + (upper ? tj1 : tj0), b, elj_e,
                                               ec_e);
            float *fk = s_fi + k * 96 + lane;
            fk[0] = __fmaf_rn(p, d.x, fk[0]);
            fk[32] = __fmaf_rn(p, d.y, fk[32]);
            fk[64] = __fmaf_rn(p, d.z, fk[64]);
            if (upper) {
                fjx.y = __fmaf_rn(-p, d.x, fjx.y);
                fjy.y = __fmaf_rn(-p, d.y, fjy.y);
                fjz.y = __fmaf_rn(-p, d.z, fjz.y);
            } else {
                fjx.x = __fmaf_rn(-p, d.x, fjx.x);
                fjy.x = __fmaf_rn(-p, d.y, fjy.x);
                fjz.x = __fmaf_rn(-p, d.z, fjz.x);
            }
        }
        if (EN) {
            elj_e += elj2.x + elj2.y;
            ec_e += ec2.x + ec2.y;
        }
        if (PRUNE && lane == 0) v.kept[j0 + e] = (unsigned short)(keep_lo | (keep_hi << 8));
        const float f0x = fjx.x, f0y = fjy.x, f0z = fjz.x, f1x = fjx.y, f1y = fjy.y, f1z = fjz.y;
        if (EN) {
            elj.add(elj_e);
            ec.add(ec_e);
        }
        // j-force reduction over the 8 i-lanes, transposed: partners ti and ti ^ 4
        // swap halves (lanes ti < 4 keep j-atom tj, lanes ti >= 4 keep tj + 4), then
        // a butterfly over the remaining 4 lanes sums one atom per lane group
        const bool upper = ti & 4;
        float kx = upper ? f1x : f0x, ky = upper ? f1y : f0y, kz = upper ? f1z : f0z;
        kx += __shfl_xor_sync(full, upper ? f0x : f1x, 4);
        ky += __shfl_xor_sync(full, upper ? f0y : f1y, 4);
        kz += __shfl_xor_sync(full, upper ? f0z : f1z, 4);
#pragma unroll
        for (int o = 1; o < 4; o <<= 1) {
            kx += __shfl_xor_sync(full, kx, o);
            ky += __shfl_xor_sync(full, ky, o);
            kz += __shfl_xor_sync(full, kz, o);
        }
        if ((ti & 3) == 0) {
            atomicAdd(&v.f[cj * NB_CL + tj + (upper ? 4 : 0)], make_float4(kx, ky, kz, 0.f));
            if (VIR) {  // the j-atom's share of sum r (x) F, from its reduced force
                const float4 xj = upper ? xj1 : xj0;
                const float ux = xj.x - org.x, uy = xj.y - org.y, uz = xj.z - org.z;
                vr[0] += ux * kx;
                vr[1] += ux * ky;
                vr[2] += ux * kz;
                vr[3] += uy * kx;
                vr[4] += uy * ky;
                vr[5] += uy * kz;
                vr[6] += uz * kx;
                vr[7] += uz * ky;
                vr[8] += uz * kz;
            }
        }
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < NB_SCL; k++) {
        float fx = s_fi[k * 96 + lane], fy = s_fi[k * 96 + 32 + lane], fz = s_fi[k * 96 + 64 + lane];
        if (VIR) {
            const float4 xi = s_xi[k * NB_CL + ti];
            const float ux = xi.x - org.x, uy = xi.y - org.y, uz = xi.z - org.z;
            vr[0] += ux * fx;
            vr[1] += ux * fy;
            vr[2] += ux * fz;
            vr[3] += uy * fx;
            vr[4] += uy * fy;
            vr[5] += uy * fz;
            vr[6] += uz * fx;
            vr[7] += uz * fy;
            vr[8] += uz * fz;
        }
        fx += __shfl_xor_sync(full, fx, 8);
        fy += __shfl_xor_sync(full, fy, 8);
        fz += __shfl_xor_sync(full, fz, 8);
        fx += __shfl_xor_sync(full, fx, 16);
        fy += __shfl_xor_sync(full, fy, 16);
        fz += __shfl_xor_sync(full, fz, 16);
        if (tj == 0) atomicAdd(&v.f[si * NB_SCA + k * NB_CL + ti], make_float4(fx, fy, fz, 0.f));
    }
}

// Warp reduction of the per-lane energy/virial accumulators (FP32; compensated
// for the energies).  Every lane ends with the warp total.
template <bool EN, bool VIR>
__device__ __forceinline__ void warp_reduce_outputs(KSum &elj, KSum &ec, float (&vr)[9]) {
    const unsigned full = 0xffffffffu;
    for (int o = 16; o > 0; o >>= 1) {
        if (EN) {
            const float a = __shfl_xor_sync(full, elj.s, o), ac = __shfl_xor_sync(full, elj.c, o);
            const float b = __shfl_xor_sync(full, ec.s, o), bc = __shfl_xor_sync(full, ec.c, o);
            elj.merge(a, ac);
            ec.merge(b, bc);
        }
        if (VIR) {
#pragma unroll
            for (int k = 0; k < 9; k++) vr[k] += __shfl_xor_sync(full, vr[k], o);
        }
    }
}

}  // namespace nbk
