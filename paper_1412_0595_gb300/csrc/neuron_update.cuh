// Per-neuron work of one time step, shared by the step kernels: Poisson
// source draw, drive event, synaptic current, Euler substeps of the HH
// equations, threshold crossing, and the decays.
#pragma once

#include "device_math.cuh"
#include "snn_internal.cuh"

namespace snn {

// Copies a population descriptor into shared memory (the calling CTA's
// threads cooperate; the caller synchronises before use).  Reading the
// per-population constants from shared memory keeps them off the global
// load path of every step.
__device__ __forceinline__ void copy_pop(DevPop* dst, const DevPop* src) {
    static_assert(sizeof(DevPop) % 4 == 0, "DevPop is copied in 4-byte words");
    const int words = (int)(sizeof(DevPop) / 4);
    for (int i = threadIdx.x; i < words; i += blockDim.x)
        reinterpret_cast<int*>(dst)[i] = reinterpret_cast<const int*>(src)[i];
}

struct NeuronState {
    float V, m, h, n, g0, g1, ie;
};

// Per-step input noise of an Izhikevich neuron: the top 20 bits of the 12
// words of three Philox draws (streams kStreamIzhNoise + 0..2), summed as
// integers (S < 12 * 2^20) and centred: z = (S - 6 * 2^20) * 2^-20, an
// Irwin-Hall approximation of a standard normal, exact in FP32.
__device__ __forceinline__ float izh_noise(PhiloxKey key, uint32_t t, uint32_t local, uint32_t tag) {
    int S = 0;
#pragma unroll
    for (uint32_t k = 0; k < 3; ++k) {
        const uint4 r = philox_4x32_10(make_uint4(local, t, tag, kStreamIzhNoise + k), key);
        S += (int)(r.x >> 12) + (int)(r.y >> 12) + (int)(r.z >> 12) + (int)(r.w >> 12);
    }
    return (float)(S - 6 * (1 << 20)) * 0x1p-20f;
}

// Per-neuron parameter draw r of an Izhikevich population (top 24 bits).
__device__ __forceinline__ float izh_r(PhiloxKey key, uint32_t local, uint32_t tag) {
    const uint4 r = philox_4x32_10(make_uint4(local, 0u, tag, kStreamIzhParam), key);
    return (float)(r.x >> 8) * 0x1p-24f;
}

// Synaptic current of the two channels from the step-start potential:
// g0 (E0 - V) + g1 (E1 - V).
template <class T>
__device__ __forceinline__ T hh_isyn(const DevPop& P, T g0, T g1, T V) {
    const T m1 = splat<T>(-1.0f);
    return vfma(g0, vfma(V, m1, splat<T>(P.E0)), vmul(g1, vfma(V, m1, splat<T>(P.E1))));
}

// Advances one neuron (population P, local index `local`) through step t.
// On entry s holds the step-start state (g0/g1 include all events delivered
// so far); on exit the step-end state with decayed conductances and drive.
// Returns whether the neuron spiked; *isyn receives I_syn of the step.
__device__ __forceinline__ bool neuron_step(const DevPop& P, PhiloxKey key, uint32_t t, int local,
                                            float hs, int n_sub, NeuronState& s, float* isyn) {
    if (P.kind == SNN_POP_SOURCE) {
        const uint4 r = philox_4x32_10(make_uint4((uint32_t)local, t, P.tag, kStreamSource), key);
        *isyn = 0.0f;
        return below(r.x, P.thr_src);
    }
    if (P.kind == SNN_POP_IZH) {
        // state: V = v, m = u, h = r (the neuron's parameter draw); the
        // synaptic input g0 + g1 is a current
        const float r = s.h;
        const float a = fmaf(P.izh[1], r, P.izh[0]), b = fmaf(P.izh[3], r, P.izh[2]);
        const float c = fmaf(P.izh[5], r * r, P.izh[4]), d = fmaf(P.izh[7], r * r, P.izh[6]);
        const float I_syn = s.g0 + s.g1;
        const float I = fmaf(P.noise, izh_noise(key, t, (uint32_t)local, P.tag), P.bias) + I_syn;
        float v = s.V;
        for (int k = 0; k < n_sub; ++k) v = fmaf(hs, fmaf(fmaf(0.04f, v, 5.0f), v, 140.0f - s.m + I), v);
        s.m = fmaf(P.dt * a, fmaf(b, v, -s.m), s.m);
        const bool spike = v >= P.v_thresh;
        if (spike) {
            v = c;
            s.m += d;
        }
        s.V = v;
        s.g0 *= P.d0;
        s.g1 *= P.d1;
        *isyn = I_syn;
        return spike;
    }
    if (P.thr_drive) {
        const uint4 r = philox_4x32_10(make_uint4((uint32_t)local, t, P.tag, kStreamDrive), key);
        if (below(r.x, P.thr_drive)) s.ie += P.drive_amp;
    }
    const float V0 = s.V;
    const float I_syn = hh_isyn<float>(P, s.g0, s.g1, V0);
    const HHConstT<float> k = hh_consts<float>(HHCell{P.gNa, P.ENa, P.gK, P.EK, P.gL, P.EL}, hs, P.hs_over_C);
    const float I_base = vadd(vadd(I_syn, s.ie), k.gLEL);
    if (n_sub == 4) {                                  // the usual count, unrolled so substeps overlap
#pragma unroll
        for (int q = 0; q < 4; ++q) hh_substep_t<float>(k, I_base, s.V, s.m, s.h, s.n);
    } else {
        for (int q = 0; q < n_sub; ++q) hh_substep_t<float>(k, I_base, s.V, s.m, s.h, s.n);
    }
    s.g0 = vmul(s.g0, P.d0);
    s.g1 = vmul(s.g1, P.d1);
    s.ie = vmul(s.ie, P.drive_dec);
    *isyn = I_syn;
    return (V0 < P.v_thresh) && (s.V >= P.v_thresh);
}

// Two neurons of one population (SoA neighbours local, local + 1), one
// thread: the HH update runs on FP32x2 operands; the other kinds step each
// neuron alone.  Bit e of the result is neuron local + e's spike.
struct NeuronPair {
    float2 V, m, h, n, g0, g1, ie;
};

__device__ __forceinline__ NeuronState pair_half(const NeuronPair& s, int e) {
    return e == 0 ? NeuronState{s.V.x, s.m.x, s.h.x, s.n.x, s.g0.x, s.g1.x, s.ie.x}
                  : NeuronState{s.V.y, s.m.y, s.h.y, s.n.y, s.g0.y, s.g1.y, s.ie.y};
}

__device__ __forceinline__ void set_pair_half(NeuronPair& s, int e, const NeuronState& h) {
    if (e == 0) { s.V.x = h.V; s.m.x = h.m; s.h.x = h.h; s.n.x = h.n; s.g0.x = h.g0; s.g1.x = h.g1; s.ie.x = h.ie; }
    else { s.V.y = h.V; s.m.y = h.m; s.h.y = h.h; s.n.y = h.n; s.g0.y = h.g0; s.g1.y = h.g1; s.ie.y = h.ie; }
}

// Per-launch constants of an HH population's pair update (held in
// registers by callers that keep a thread on one population).
struct HHPairConsts {
    HHConstT<float2> k;
    float2 E0, E1, d0, d1, ddec;
    float v_thresh, drive_amp;
    unsigned long long thr_drive;
    uint32_t tag;
};

__device__ __forceinline__ HHPairConsts hh_pair_consts(const DevPop& P, float hs) {
    HHPairConsts c;
    c.k = hh_consts<float2>(HHCell{P.gNa, P.ENa, P.gK, P.EK, P.gL, P.EL}, hs, P.hs_over_C);
    c.E0 = splat<float2>(P.E0);
    c.E1 = splat<float2>(P.E1);
    c.d0 = splat<float2>(P.d0);
    c.d1 = splat<float2>(P.d1);
    c.ddec = splat<float2>(P.drive_dec);
    c.v_thresh = P.v_thresh;
    c.drive_amp = P.drive_amp;
    c.thr_drive = P.thr_drive;
    c.tag = P.tag;
    return c;
}

// The drive events of neurons local and local + 1 at step t (bit e: one
// event for neuron local + e).
__device__ __forceinline__ unsigned hh_drive_pair(const HHPairConsts& c, PhiloxKey key, uint32_t t, int local) {
    if (!c.thr_drive) return 0u;
    const uint4 r0 = philox_4x32_10(make_uint4((uint32_t)local, t, c.tag, kStreamDrive), key);
    const uint4 r1 = philox_4x32_10(make_uint4((uint32_t)local + 1u, t, c.tag, kStreamDrive), key);
    return (below(r0.x, c.thr_drive) ? 1u : 0u) | (below(r1.x, c.thr_drive) ? 2u : 0u);
}

// The HH update of neurons local and local + 1 through one step (the pair
// form of neuron_step's HH branch, identical per element), given the step's
// drive events and the rates at the step-start potentials (both depend on
// nothing a pull delivers, so a caller may compute them early).
__device__ __forceinline__ unsigned hh_step_pair_given(const HHPairConsts& c, unsigned drive, const RatesT<float2>& r0,
                                                       int n_sub, NeuronPair& s, float2* isyn) {
    if (drive & 1u) s.ie.x += c.drive_amp;
    if (drive & 2u) s.ie.y += c.drive_amp;
    const float2 V0 = s.V;
    const float2 m1 = splat<float2>(-1.0f);
    const float2 I_syn = vfma(s.g0, vfma(V0, m1, c.E0), vmul(s.g1, vfma(V0, m1, c.E1)));
    const float2 I_base = vadd(vadd(I_syn, s.ie), c.k.gLEL);
    hh_substep_r<float2>(c.k, r0, I_base, s.V, s.m, s.h, s.n);
    if (n_sub == 4) {
#pragma unroll
        for (int q = 1; q < 4; ++q) hh_substep_t<float2>(c.k, I_base, s.V, s.m, s.h, s.n);
    } else {
        for (int q = 1; q < n_sub; ++q) hh_substep_t<float2>(c.k, I_base, s.V, s.m, s.h, s.n);
    }
    s.g0 = vmul(s.g0, c.d0);
    s.g1 = vmul(s.g1, c.d1);
    s.ie = vmul(s.ie, c.ddec);
    *isyn = I_syn;
    return ((V0.x < c.v_thresh) && (s.V.x >= c.v_thresh) ? 1u : 0u) |
           ((V0.y < c.v_thresh) && (s.V.y >= c.v_thresh) ? 2u : 0u);
}

__device__ __forceinline__ unsigned hh_step_pair(const HHPairConsts& c, PhiloxKey key, uint32_t t, int local, int n_sub,
                                                 NeuronPair& s, float2* isyn) {
    const unsigned drive = hh_drive_pair(c, key, t, local);
    return hh_step_pair_given(c, drive, hh_rates(s.V), n_sub, s, isyn);
}

__device__ __forceinline__ unsigned neuron_step_pair(const DevPop& P, PhiloxKey key, uint32_t t, int local,
                                                     float hs, int n_sub, NeuronPair& s, float2* isyn) {
    if (P.kind != SNN_POP_HH) {
        unsigned spk = 0;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            NeuronState h = pair_half(s, e);
            float is;
            if (neuron_step(P, key, t, local + e, hs, n_sub, h, &is)) spk |= 1u << e;
            set_pair_half(s, e, h);
            if (e == 0) isyn->x = is; else isyn->y = is;
        }
        return spk;
    }
    return hh_step_pair(hh_pair_consts(P, hs), key, t, local, n_sub, s, isyn);
}

}  // namespace snn
