// Device-side building blocks: the Philox4x32-10 counter-based generator,
// FP32 Traub-Miles HH rates and one forward-Euler substep, and the
// acquire/release accesses used by the bounded device-side waits.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace snn {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64-bit
// multiplies whose halves are cross-xored with the other two words and the
// round key; the key advances by the golden-ratio / sqrt(3) Weyl increments.
// ---------------------------------------------------------------------------
struct PhiloxKey {
    uint32_t k0, k1;
};

__device__ __forceinline__ uint4 philox_4x32_10(uint4 x, PhiloxKey key) {
    constexpr uint32_t kMulA = 0xD2511F53u, kMulB = 0xCD9E8D57u;
    constexpr uint32_t kWeylA = 0x9E3779B9u, kWeylB = 0xBB67AE85u;
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t a_hi = __umulhi(kMulA, x.x), a_lo = kMulA * x.x;
        const uint32_t b_hi = __umulhi(kMulB, x.z), b_lo = kMulB * x.z;
        x = make_uint4(b_hi ^ x.y ^ key.k0, b_lo, a_hi ^ x.w ^ key.k1, a_lo);
        key.k0 += kWeylA;
        key.k1 += kWeylB;
    }
    return x;
}

// Bernoulli event: the 32-bit draw is below the integer threshold round(p*2^32).
__device__ __forceinline__ bool below(uint32_t u, unsigned long long thr) {
    return (unsigned long long)u < thr;
}

// ---------------------------------------------------------------------------
// Traub-Miles HH in FP32 (V in mV, t in ms, g in nS, C in pF, I in pA).
// ---------------------------------------------------------------------------
// x / (exp(x) - 1), continuous through x = 0 (removable singularity of the
// linoid rates); the series 1 - x/2 + x^2/12 is exact to FP32 for |x| < 1e-3.
__device__ __forceinline__ float linoid(float x) {
    if (fabsf(x) < 1e-3f) return fmaf(x, fmaf(x, 1.0f / 12.0f, -0.5f), 1.0f);
    return x / expm1f(x);
}

struct HHCell {
    float gNa, ENa, gK, EK, gL, EL;
};

struct HHRates {
    float am, bm, ah, bh, an, bn;
};

// 2^x and 1/x on the special-function unit (PTX ex2.approx.ftz.f32 and
// rcp.approx.ftz.f32: relative error about 2^-22, subnormals flushed).
__device__ __forceinline__ float ex2_fast(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_fast(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ---------------------------------------------------------------------------
// One- and two-neuron arithmetic.  The HH update is written once, over T =
// float (one neuron) or float2 (two neurons of one population, one thread).
// For float2 the FP32x2 instructions of sm_100 and later (FFMA2, FADD2,
// FMUL2) apply the FP32 operation, with its single rounding, to both halves:
// per element exactly fmaf / __fadd_rn / __fmul_rn, so both forms give the
// same bits.  Explicit _rn forms keep the compiler from contracting a
// multiply and an add into a fused one in one form and not the other.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float vex2(float a) { return ex2_fast(a); }
__device__ __forceinline__ float2 vex2(float2 a) { return make_float2(ex2_fast(a.x), ex2_fast(a.y)); }
__device__ __forceinline__ float vrcp(float a) { return rcp_fast(a); }
__device__ __forceinline__ float2 vrcp(float2 a) { return make_float2(rcp_fast(a.x), rcp_fast(a.y)); }
__device__ __forceinline__ float vneg(float a) { return -a; }
__device__ __forceinline__ float2 vneg(float2 a) { return make_float2(-a.x, -a.y); }

template <class T> __device__ __forceinline__ T splat(float c);
template <> __device__ __forceinline__ float splat<float>(float c) { return c; }
template <> __device__ __forceinline__ float2 splat<float2>(float c) { return make_float2(c, c); }

template <class T> struct RatesT {
    T am, bm, ah, bh, an, bn;
};

// Per-element helpers of the near-singularity handling.
struct Near1 {
    bool x, y, z;
};
struct Near2 {
    Near1 e0, e1;
};
__device__ __forceinline__ Near1 near_flags(float xs, float ys, float zs) {
    // |x| < 0.05 <=> |1.28 x| < 0.064, |y| < 0.05 <=> |1.4 y| < 0.07, |z| < 0.05 <=> |0.16 z| < 0.008
    return Near1{fabsf(xs) < 0.064f, fabsf(ys) < 0.07f, fabsf(zs) < 0.008f};
}
__device__ __forceinline__ Near1 near_of(float xs, float ys, float zs) { return near_flags(xs, ys, zs); }
__device__ __forceinline__ Near2 near_of(float2 xs, float2 ys, float2 zs) {
    return Near2{near_flags(xs.x, ys.x, zs.x), near_flags(xs.y, ys.y, zs.y)};
}
__device__ __forceinline__ bool any_near(const Near1& f) { return f.x | f.y | f.z; }
__device__ __forceinline__ bool any_near(const Near2& f) { return any_near(f.e0) | any_near(f.e1); }
__device__ __forceinline__ float sel_x(const Near1& f, float a, float b) { return f.x ? a : b; }
__device__ __forceinline__ float sel_y(const Near1& f, float a, float b) { return f.y ? a : b; }
__device__ __forceinline__ float sel_z(const Near1& f, float a, float b) { return f.z ? a : b; }
__device__ __forceinline__ float2 sel_x(const Near2& f, float2 a, float2 b) {
    return make_float2(f.e0.x ? a.x : b.x, f.e1.x ? a.y : b.y);
}
__device__ __forceinline__ float2 sel_y(const Near2& f, float2 a, float2 b) {
    return make_float2(f.e0.y ? a.x : b.x, f.e1.y ? a.y : b.y);
}
__device__ __forceinline__ float2 sel_z(const Near2& f, float2 a, float2 b) {
    return make_float2(f.e0.z ? a.x : b.x, f.e1.z ? a.y : b.y);
}

// Traub-Miles rates, one or two neurons.  The four denominators of the
// rational rates, a = exp(x) - 1, b = exp(y) - 1, c = exp(-5) - exp(y) and
// d = exp(y) + 1 (E = exp(y) also serves beta_h = 4 E / (E + 1) and, with
// exp(z) = exp(-5) / E, alpha_n = 0.16 z E / (exp(-5) - E)), share one
// reciprocal r = 1/(a b c d): 1/a = b (c d r), 1/b = a (c d r),
// 1/c = d (a b r), 1/d = c (a b r) -- four exponentials and one reciprocal.
// Near a removable singularity (linoid argument within 0.05 of zero, where
// exp(x) - 1 would lose digits to cancellation) the rate is the series
// k (1 - x/2 + x^2/12) (the omitted x^4/720 is below 1e-8 relative there) and
// its denominator enters the product as 1, so the other rates, in which it
// cancels, stay exact and nothing divides by zero.  Outside those windows the
// cancellation error is below 5e-6 relative.  The product overflows FP32
// only above about +120 mV (the rates then turn NaN, as the separate
// reciprocals do from about +390 mV), far outside the Euler dynamics of a
// stable run.  The windows are rare (an upstroke crosses each in about one
// substep), so a warp takes the careful form only when one of its lanes is in
// one; both forms give the same value outside the windows.
template <class T, bool kCareful>
__device__ __forceinline__ RatesT<T> hh_rates_form(T V, T xs, T ys, T zs, T Em, T E) {
    constexpr float kExpM5 = 6.737946999085467e-3f;
    constexpr float L = 1.4426950408889634f;
    RatesT<T> r;
    r.ah = vex2(vfma(V, splat<T>(-L / 18.0f), splat<T>(-48.0f * L / 18.0f - 2.965784284662087f)));   // + log2 0.128
    r.bn = vex2(vfma(V, splat<T>(-L / 40.0f), splat<T>(-55.0f * L / 40.0f - 1.0f)));                 // + log2 0.5
    T a = vadd(Em, splat<T>(-1.0f));
    T b = vadd(E, splat<T>(-1.0f));
    T c = vfma(E, splat<T>(-1.0f), splat<T>(kExpM5));
    const T d = vadd(E, splat<T>(1.0f));
    const auto nf = near_of(xs, ys, zs);
    if (kCareful) {
        a = sel_x(nf, splat<T>(1.0f), a);
        b = sel_y(nf, splat<T>(1.0f), b);
        c = sel_z(nf, splat<T>(1.0f), c);
    }
    const T ab = vmul(a, b), cd = vmul(c, d);
    const T rr = vrcp(vmul(ab, cd));
    const T abr = vmul(ab, rr), cdr = vmul(cd, rr);
    r.am = vmul(xs, vmul(b, cdr));
    r.bm = vmul(ys, vmul(a, cdr));
    r.an = vmul(vmul(zs, E), vmul(d, abr));
    r.bh = vmul(vmul(E, splat<T>(4.0f)), vmul(c, abr));
    if (kCareful) {
        // k L(x) as a quadratic in xs = k x: k - xs/2 + xs^2 / (12 k); for
        // alpha_n, E cancels: 0.16 z E / (exp(-5) - E) = 0.16 L(z)
        const T sm = vfma(xs, vfma(xs, splat<T>(1.0f / (12.0f * 1.28f)), splat<T>(-0.5f)), splat<T>(1.28f));
        const T sb = vfma(ys, vfma(ys, splat<T>(1.0f / (12.0f * 1.4f)), splat<T>(-0.5f)), splat<T>(1.4f));
        const T sn = vfma(zs, vfma(zs, splat<T>(1.0f / (12.0f * 0.16f)), splat<T>(-0.5f)), splat<T>(0.16f));
        r.am = sel_x(nf, sm, r.am);
        r.bm = sel_y(nf, sb, r.bm);
        r.an = sel_z(nf, sn, r.an);
    }
    return r;
}

__device__ __forceinline__ unsigned active_lanes() { return __activemask(); }

template <class T>
__device__ __forceinline__ RatesT<T> hh_rates_t(T V) {
    constexpr float L = 1.4426950408889634f;
    const T xs = vfma(V, splat<T>(-0.25f * 1.28f), splat<T>(-13.0f * 1.28f));   // 1.28 x, x = (-52 - V)/4
    const T ys = vfma(V, splat<T>(0.2f * 1.4f), splat<T>(5.0f * 1.4f));         // 1.4 y,  y = (V + 25)/5
    const T zs = vfma(V, splat<T>(-0.2f * 0.16f), splat<T>(-10.0f * 0.16f));    // 0.16 z, z = (-50 - V)/5
    const T Em = vex2(vfma(V, splat<T>(-0.25f * L), splat<T>(-13.0f * L)));
    const T E = vex2(vfma(V, splat<T>(0.2f * L), splat<T>(5.0f * L)));
    // warp-uniform choice of the form (every lane of the warp takes the same branch)
    if (__any_sync(active_lanes(), any_near(near_of(xs, ys, zs))))
        return hh_rates_form<T, true>(V, xs, ys, zs, Em, E);
    return hh_rates_form<T, false>(V, xs, ys, zs, Em, E);
}

__device__ __forceinline__ HHRates hh_rates(float V) {
    const RatesT<float> f = hh_rates_t<float>(V);
    return HHRates{f.am, f.bm, f.ah, f.bh, f.an, f.bn};
}

__device__ __forceinline__ RatesT<float2> hh_rates(float2 V) { return hh_rates_t<float2>(V); }

__device__ __forceinline__ RatesT<float> as_rates_t(const HHRates& r) {
    return RatesT<float>{r.am, r.bm, r.ah, r.bh, r.an, r.bn};
}
__device__ __forceinline__ RatesT<float2> as_rates_t(const RatesT<float2>& r) { return r; }

// Per-step constants of one population's HH update, as one- or two-neuron
// operands: the currents as g (E - V) = fma(-g, V, g E).
template <class T>
struct HHConstT {
    T ngL, ngK, gKEK, ngNa, gNaENa, hs, hs_over_C, gLEL;
};

template <class T>
__device__ __forceinline__ HHConstT<T> hh_consts(const HHCell& c, float hs, float hs_over_C) {
    return HHConstT<T>{splat<T>(-c.gL), splat<T>(-c.gK), splat<T>(c.gK * c.EK), splat<T>(-c.gNa),
                       splat<T>(c.gNa * c.ENa), splat<T>(hs), splat<T>(hs_over_C), splat<T>(c.gL * c.EL)};
}

// One forward-Euler substep with every right-hand side at the substep start,
// given the rates at V; I_base = I_syn + I_ext + gL EL (held over the
// substeps).
//   V += hs/C (I_base - gL V - gK n^4 (V - EK) - gNa m^3 h (V - ENa))
//   x += hs (alpha_x - (alpha_x + beta_x) x),  x in {m, h, n}
template <class T>
__device__ __forceinline__ void hh_substep_r(const HHConstT<T>& k, const RatesT<T>& r, T I_base, T& V, T& m, T& h,
                                             T& n) {
    const T m3h = vmul(vmul(vmul(m, m), m), h);
    const T n2 = vmul(n, n);
    const T n4 = vmul(n2, n2);
    T I = vfma(k.ngL, V, I_base);
    I = vfma(n4, vfma(k.ngK, V, k.gKEK), I);
    I = vfma(m3h, vfma(k.ngNa, V, k.gNaENa), I);
    m = vfma(k.hs, vfma(vneg(vadd(r.am, r.bm)), m, r.am), m);
    h = vfma(k.hs, vfma(vneg(vadd(r.ah, r.bh)), h, r.ah), h);
    n = vfma(k.hs, vfma(vneg(vadd(r.an, r.bn)), n, r.an), n);
    V = vfma(k.hs_over_C, I, V);
}

template <class T>
__device__ __forceinline__ void hh_substep_t(const HHConstT<T>& k, T I_base, T& V, T& m, T& h, T& n) {
    hh_substep_r<T>(k, as_rates_t(hh_rates(V)), I_base, V, m, h, n);
}

// One-neuron form used by the graded network's forward and adjoint passes
// (identical arithmetic to the template above).
__device__ __forceinline__ void hh_substep(const HHCell& c, float hs, float hs_over_C, float I_in,
                                           float& V, float& m, float& h, float& n) {
    const HHConstT<float> k = hh_consts<float>(c, hs, hs_over_C);
    hh_substep_t<float>(k, vadd(I_in, k.gLEL), V, m, h, n);
}

// Steady-state gating alpha / (alpha + beta) at V.
__device__ __forceinline__ void hh_steady(float V, float& m, float& h, float& n) {
    const float am = 1.28f * linoid((-52.0f - V) * 0.25f);
    const float bm = 1.4f * linoid((V + 25.0f) * 0.2f);
    const float ah = 0.128f * expf((-48.0f - V) * (1.0f / 18.0f));
    const float bh = 4.0f / (expf((-25.0f - V) * 0.2f) + 1.0f);
    const float an = 0.16f * linoid((-50.0f - V) * 0.2f);
    const float bn = 0.5f * expf((-55.0f - V) * 0.025f);
    m = am / (am + bm);
    h = ah / (ah + bh);
    n = an / (an + bn);
}

// ---------------------------------------------------------------------------
// Memory-model helpers for flags shared between CTAs.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void st_release_u32(unsigned int* p, unsigned int v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

}  // namespace snn
