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
    if (P.thr_drive) {
        const uint4 r = philox_4x32_10(make_uint4((uint32_t)local, t, P.tag, kStreamDrive), key);
        if (below(r.x, P.thr_drive)) s.ie += P.drive_amp;
    }
    const float V0 = s.V;
    const float I_syn = s.g0 * (P.E0 - V0) + s.g1 * (P.E1 - V0);
    const float I_in = I_syn + s.ie;
    const HHCell cell{P.gNa, P.ENa, P.gK, P.EK, P.gL, P.EL};
    for (int k = 0; k < n_sub; ++k) hh_substep(cell, hs, P.hs_over_C, I_in, s.V, s.m, s.h, s.n);
    s.g0 *= P.d0;
    s.g1 *= P.d1;
    s.ie *= P.drive_dec;
    *isyn = I_syn;
    return (V0 < P.v_thresh) && (s.V >= P.v_thresh);
}

}  // namespace snn
