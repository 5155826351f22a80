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
    const float I_syn = s.g0 * (P.E0 - V0) + s.g1 * (P.E1 - V0);
    const float I_in = I_syn + s.ie;
    const HHCell cell{P.gNa, P.ENa, P.gK, P.EK, P.gL, P.EL};
    if (n_sub == 4) {                                  // the usual count, unrolled so substeps overlap
#pragma unroll
        for (int k = 0; k < 4; ++k) hh_substep(cell, hs, P.hs_over_C, I_in, s.V, s.m, s.h, s.n);
    } else {
        for (int k = 0; k < n_sub; ++k) hh_substep(cell, hs, P.hs_over_C, I_in, s.V, s.m, s.h, s.n);
    }
    s.g0 *= P.d0;
    s.g1 *= P.d1;
    s.ie *= P.drive_dec;
    *isyn = I_syn;
    return (V0 < P.v_thresh) && (s.V >= P.v_thresh);
}

}  // namespace snn
