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

// Taylor series of x / (exp(x) - 1) about 0 to x^4 (Bernoulli numbers
// B1 = -1/2, B2 = 1/6, B4 = -1/30): 1 - x/2 + x^2/12 - x^4/720; the first
// omitted term is x^6/30240, below 2e-11 for |x| < 0.1.
__device__ __forceinline__ float linoid_series(float x) {
    const float x2 = x * x;
    return fmaf(x2, fmaf(x2, -1.0f / 720.0f, 1.0f / 12.0f), fmaf(-0.5f, x, 1.0f));
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

// Traub-Miles rates (1/ms, V in mV):
//   alpha_m = 1.28 x / (exp(x) - 1), x = (-52 - V)/4     beta_m = 1.4 y / (exp(y) - 1), y = (V + 25)/5
//   alpha_h = 0.128 exp((-48 - V)/18)                   beta_h = 4 / (exp(-y) + 1)
//   alpha_n = 0.16 z / (exp(z) - 1), z = (-50 - V)/5     beta_n = 0.5 exp((-55 - V)/40)
//
// Careful form, one neuron: four exponentials and a reciprocal per rational
// rate.  E = exp(y) serves three rates: beta_h = 4 E / (E + 1) and, with
// exp(z) = exp(-5) / E, alpha_n = 0.16 z E / (exp(-5) - E).  Linoid rates
// switch to the series for |argument| < 0.1, where exp(x) - 1 loses digits
// to cancellation.
__device__ __forceinline__ HHRates hh_rates_careful(float V) {
    constexpr float L = 1.4426950408889634f;             // log2(e)
    constexpr float kExpM5 = 6.737946999085467e-3f;     // exp(-5)
    const float xs = fmaf(V, -0.25f * 1.28f, -13.0f * 1.28f);   // 1.28 x
    const float ys = fmaf(V, 0.2f * 1.4f, 5.0f * 1.4f);         // 1.4 y
    const float zs = fmaf(V, -0.2f * 0.16f, -10.0f * 0.16f);    // 0.16 z
    const float Em = ex2_fast(fmaf(V, -0.25f * L, -13.0f * L));
    const float E = ex2_fast(fmaf(V, 0.2f * L, 5.0f * L));
    HHRates r;
    r.ah = ex2_fast(fmaf(V, -L / 18.0f, -48.0f * L / 18.0f - 2.965784284662087f));   // + log2 0.128
    r.bn = ex2_fast(fmaf(V, -L / 40.0f, -55.0f * L / 40.0f - 1.0f));                 // + log2 0.5
    r.am = xs * rcp_fast(Em - 1.0f);
    r.bm = ys * rcp_fast(E - 1.0f);
    r.an = zs * E * rcp_fast(kExpM5 - E);
    const float x = fmaf(V, -0.25f, -13.0f), y = fmaf(V, 0.2f, 5.0f), z = fmaf(V, -0.2f, -10.0f);
    if (fabsf(x) < 0.1f) r.am = 1.28f * linoid_series(x);
    if (fabsf(y) < 0.1f) r.bm = 1.4f * linoid_series(y);
    if (fabsf(z) < 0.1f) r.an = 0.16f * linoid_series(z);
    r.bh = 4.0f * E * rcp_fast(E + 1.0f);
    return r;
}

// The careful form covers -52.4 < V < -24.5 mV (every linoid argument within
// 0.1 of its singularity lies there); outside it the fast form below applies.
__device__ __forceinline__ bool rates_need_care(float V) { return fabsf(V + 38.45f) < 13.95f; }

// Fast form: the four denominators a = exp(x) - 1, b = exp(y) - 1,
// c = exp(-5) - exp(y), d = exp(y) + 1 share one reciprocal r = 1/(a b c d),
// and 1/a = b (c d r), 1/b = a (c d r), 1/c = d (a b r), 1/d = c (a b r):
// four exponentials and one reciprocal instead of four and four.  Outside
// [-52.4, -24.5] mV no denominator is near zero; the product overflows FP32
// only above about +120 mV (the rates then turn NaN, as the separate
// reciprocals do from about +390 mV), far outside the Euler dynamics of a
// stable run.
template <class T>
__device__ __forceinline__ RatesT<T> hh_rates_fast(T V) {
    constexpr float L = 1.4426950408889634f;
    constexpr float kExpM5 = 6.737946999085467e-3f;
    const T xs = vfma(V, splat<T>(-0.25f * 1.28f), splat<T>(-13.0f * 1.28f));
    const T ys = vfma(V, splat<T>(0.2f * 1.4f), splat<T>(5.0f * 1.4f));
    const T zs = vfma(V, splat<T>(-0.2f * 0.16f), splat<T>(-10.0f * 0.16f));
    const T Em = vex2(vfma(V, splat<T>(-0.25f * L), splat<T>(-13.0f * L)));
    const T E = vex2(vfma(V, splat<T>(0.2f * L), splat<T>(5.0f * L)));
    RatesT<T> r;
    r.ah = vex2(vfma(V, splat<T>(-L / 18.0f), splat<T>(-48.0f * L / 18.0f - 2.965784284662087f)));
    r.bn = vex2(vfma(V, splat<T>(-L / 40.0f), splat<T>(-55.0f * L / 40.0f - 1.0f)));
    const T a = vadd(Em, splat<T>(-1.0f));
    const T b = vadd(E, splat<T>(-1.0f));
    const T c = vfma(E, splat<T>(-1.0f), splat<T>(kExpM5));
    const T d = vadd(E, splat<T>(1.0f));
    const T ab = vmul(a, b), cd = vmul(c, d);
    const T rr = vrcp(vmul(ab, cd));
    const T abr = vmul(ab, rr), cdr = vmul(cd, rr);
    r.am = vmul(xs, vmul(b, cdr));
    r.bm = vmul(ys, vmul(a, cdr));
    r.an = vmul(vmul(zs, E), vmul(d, abr));
    r.bh = vmul(vmul(E, splat<T>(4.0f)), vmul(c, abr));
    return r;
}

__device__ __forceinline__ HHRates hh_rates(float V) {
    if (rates_need_care(V)) return hh_rates_careful(V);
    const RatesT<float> f = hh_rates_fast<float>(V);
    return HHRates{f.am, f.bm, f.ah, f.bh, f.an, f.bn};
}

__device__ __forceinline__ RatesT<float2> hh_rates(float2 V) {
    RatesT<float2> r = hh_rates_fast<float2>(V);
    if (rates_need_care(V.x)) {
        const HHRates c = hh_rates_careful(V.x);
        r.am.x = c.am; r.bm.x = c.bm; r.ah.x = c.ah; r.bh.x = c.bh; r.an.x = c.an; r.bn.x = c.bn;
    }
    if (rates_need_care(V.y)) {
        const HHRates c = hh_rates_careful(V.y);
        r.am.y = c.am; r.bm.y = c.bm; r.ah.y = c.ah; r.bh.y = c.bh; r.an.y = c.an; r.bn.y = c.bn;
    }
    return r;
}

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

// One forward-Euler substep with every right-hand side at the substep start;
// I_base = I_syn + I_ext + gL EL (held over the substeps).
//   V += hs/C (I_base - gL V - gK n^4 (V - EK) - gNa m^3 h (V - ENa))
//   x += hs (alpha_x - (alpha_x + beta_x) x),  x in {m, h, n}
template <class T>
__device__ __forceinline__ void hh_substep_t(const HHConstT<T>& k, T I_base, T& V, T& m, T& h, T& n) {
    const RatesT<T> r = as_rates_t(hh_rates(V));
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
