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

// Traub-Miles rates at V with four hardware exponentials and four
// reciprocals.  Algebraic identities used (exact in real arithmetic):
//   E = exp((V + 25)/5) serves beta_m = 1.4 y / (E - 1), y = (V + 25)/5,
//   beta_h = 4 / (1/E + 1) = 4 E / (E + 1), and
//   alpha_n = 0.16 z / (exp(z) - 1) with exp(z) = exp(-5) / E, z = (-50 - V)/5,
//   so alpha_n = 0.16 z E / (exp(-5) - E).
// Linoid rates switch to the series for |argument| < 0.1, where exp(x) - 1
// would lose digits to cancellation.
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

__device__ __forceinline__ HHRates hh_rates(float V) {
    constexpr float L = 1.4426950408889634f;             // log2(e)
    constexpr float kExpM5 = 6.737946999085467e-3f;     // exp(-5)
    // every argument is one fused multiply-add of V; the rate constants
    // 1.28, 1.4 and 0.16 are folded into the linear factors, 0.128 and 0.5
    // into the exponents (log2 0.128 and log2 0.5 = -1)
    const float xs = fmaf(V, -0.25f * 1.28f, -13.0f * 1.28f);   // 1.28 (-52 - V)/4
    const float ys = fmaf(V, 0.2f * 1.4f, 5.0f * 1.4f);         // 1.4 (V + 25)/5
    const float zs = fmaf(V, -0.2f * 0.16f, -10.0f * 0.16f);    // 0.16 (-50 - V)/5
    const float Em = ex2_fast(fmaf(V, -0.25f * L, -13.0f * L));
    const float E = ex2_fast(fmaf(V, 0.2f * L, 5.0f * L));
    HHRates r;
    r.ah = ex2_fast(fmaf(V, -L / 18.0f, -48.0f * L / 18.0f - 2.965784284662087f));
    r.bn = ex2_fast(fmaf(V, -L / 40.0f, -55.0f * L / 40.0f - 1.0f));
    r.am = xs * rcp_fast(Em - 1.0f);
    r.bm = ys * rcp_fast(E - 1.0f);
    r.an = zs * E * rcp_fast(kExpM5 - E);
    // near the removable singularities exp(x) - 1 cancels: use the series
    const bool near = (fabsf(xs) < 0.1f * 1.28f) | (fabsf(ys) < 0.1f * 1.4f) | (fabsf(zs) < 0.1f * 0.16f);
    if (near) {
        const float x = fmaf(V, -0.25f, -13.0f), y = fmaf(V, 0.2f, 5.0f), z = fmaf(V, -0.2f, -10.0f);
        if (fabsf(x) < 0.1f) r.am = 1.28f * linoid_series(x);
        if (fabsf(y) < 0.1f) r.bm = 1.4f * linoid_series(y);
        if (fabsf(z) < 0.1f) r.an = 0.16f * linoid_series(z);
    }
    r.bh = 4.0f * E * rcp_fast(E + 1.0f);
    return r;
}

// One forward-Euler substep with every right-hand side at the substep start.
// The currents are arranged as fused multiply-adds: g (V - E) = fma(g, V, -g E)
// and dx/dt = alpha - (alpha + beta) x.
__device__ __forceinline__ void hh_substep(const HHCell& c, float hs, float hs_over_C, float I_in,
                                           float& V, float& m, float& h, float& n) {
    const HHRates r = hh_rates(V);
    const float m3h = m * m * m * h;
    const float n2 = n * n;
    float I = fmaf(-c.gL, V, fmaf(c.gL, c.EL, I_in));
    I = fmaf(-(n2 * n2), fmaf(c.gK, V, -c.gK * c.EK), I);
    I = fmaf(-m3h, fmaf(c.gNa, V, -c.gNa * c.ENa), I);
    const float dm = fmaf(-(r.am + r.bm), m, r.am);
    const float dh = fmaf(-(r.ah + r.bh), h, r.ah);
    const float dn = fmaf(-(r.an + r.bn), n, r.an);
    V = fmaf(hs_over_C, I, V);
    m = fmaf(hs, dm, m);
    h = fmaf(hs, dh, h);
    n = fmaf(hs, dn, n);
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
