// Differentiable form: graded-synapse HH network, forward and discrete adjoint.
//
// Forward step (one per time step, two launches):
//   k_graded_spmv    G_q[j] = sum_i w_ij r_i for every graded projection q,
//                    pulled over the transposed (post-major) copy of the
//                    compressed rows: no atomics, a fixed summation order, so
//                    a recomputed step is bit-identical to the first pass;
//   k_graded_neuron  I_syn = sum_q s_q (E_q - V) G_q, drive events, Euler
//                    substeps, drive decay, output filter y += a (V - y)
//                    (recorded into y_out), and the next release
//                    r = 1 / (1 + exp((v_thr - V) / slope)).
// Adjoint (per checkpoint segment of K steps, in reverse):
//   the segment is recomputed from its checkpoint with the same two kernels,
//   storing step-start states, releases and G;
//   k_graded_reverse back through the filter (seeded by the caller's dL/dy),
//                    the substeps (recomputed in
//                    registers, analytic rate derivatives) and the synaptic
//                    current: state adjoints, dL/dG_q = mu s_q (E_q - V), and
//                    dL/ds_q partial sums;
//   k_graded_gather  dL/dV_i += r'_i sum_q sum_k w_ik dL/dG_q[k] over the
//                    compressed row of i (pre-synaptic path);
//   k_graded_sddmm   after the segment: dL/dw_ik += sum_t r_i(t) dL/dG_q[k](t),
//                    with dL/dG stored post-major and time-contiguous so each
//                    synapse reads K consecutive floats.
#include "device_math.cuh"
#include "snn_internal.cuh"
#include "tc_common.cuh"

namespace snn {

namespace {

constexpr int kThreads = 256;
constexpr int kNeuronThreads = 64;     // per-neuron kernels: small CTAs, so 20,000 neurons reach every SM

__device__ __forceinline__ float release(float V, float thr, float inv_slope) {
    return 1.0f / (1.0f + __expf((thr - V) * inv_slope));
}

// d/dx [x / (exp(x) - 1)]: series (Bernoulli numbers) for |x| < 0.5, else the
// closed form (e - 1 - x e) / (e - 1)^2 with e = exp(x).
__device__ __forceinline__ float dlinoid(float x, float e) {
    if (fabsf(x) < 0.5f) {
        const float x2 = x * x;
        return fmaf(x, fmaf(x2, fmaf(x2, fmaf(x2, -1.0f / 151200.0f, 1.0f / 5040.0f), -1.0f / 180.0f),
                            1.0f / 6.0f), -0.5f);
    }
    const float em = e - 1.0f;
    return __fdividef(em - x * e, em * em);
}

struct HHDerivs {
    float am, bm, ah, bh, an, bn;
};

// Derivatives in V of the rates of hh_rates (same identities).
__device__ __forceinline__ HHDerivs hh_rate_derivs(float V, const HHRates& r) {
    constexpr float kLog2e = 1.4426950408889634f;
    constexpr float kExpM5 = 6.737946999085467e-3f;
    const float x = (-52.0f - V) * 0.25f;
    const float y = (V + 25.0f) * 0.2f;
    const float z = (-50.0f - V) * 0.2f;
    const float Em = ex2_fast(x * kLog2e);
    const float E = ex2_fast(y * kLog2e);
    const float Ez = kExpM5 * rcp_fast(E);
    HHDerivs d;
    d.am = 1.28f * dlinoid(x, Em) * -0.25f;
    d.bm = 1.4f * dlinoid(y, E) * 0.2f;
    d.an = 0.16f * dlinoid(z, Ez) * -0.2f;
    d.ah = -r.ah * (1.0f / 18.0f);
    const float e1 = E + 1.0f;
    d.bh = __fdividef(0.8f * E, e1 * e1);
    d.bn = -r.bn * 0.025f;
    return d;
}

// Synaptic current of neuron `local` of population p from the G vector.
__device__ __forceinline__ float graded_isyn(const GradedArgs& a, int pop, int local, float V, float* dI_dV) {
    float isyn = 0.0f, d = 0.0f;
    const int b = a.in_begin[pop], e = a.in_begin[pop + 1];
    for (int k = b; k < e; ++k) {
        const GradProj& q = a.gprojs[a.in_list[k]];
        const float G = a.G[q.g_off + local];
        isyn += q.scale * (q.E - V) * G;
        d -= q.scale * G;
    }
    *dI_dV = d;
    return isyn;
}

constexpr int kStagedThreads = 1024;              // staged kernels: one CTA per SM
constexpr size_t kStageMaxBytes = 200 * 1024;      // largest gathered vector held in shared memory

// x[i]: from shared memory when the gathered vector is staged there (its
// random reads then cost bank conflicts instead of one L1 wavefront each),
// else through the read-only path.
template <bool kShared>
__device__ __forceinline__ float gather(const float* x, int32_t i) {
    if constexpr (kShared) return x[i];
    else return __ldg(x + i);
}

// sum over k in [b, e) of w[k] x[idx[k]] by one warp: 16-byte loads of 4
// consecutive synapses per lane, four 128-synapse blocks in flight per
// iteration (128 B per lane), one partial sum per block.  w and idx are
// padded so loads that start before e stay inside the allocation; the
// synapse arrays are streamed (evict-first).  The order of the sums is fixed,
// so a recomputed step is bit-identical.
template <bool kShared>
__device__ __forceinline__ float lane_dot(const float* w, const int32_t* idx, const float* x, int64_t b,
                                          int64_t e, int lane) {
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (int64_t k0 = (b & ~int64_t(3)) + 4 * lane; k0 < e; k0 += 512) {
        float4 wv[4];
        int4 iv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t k = k0 + 128 * u;
            if (k < e) {
                wv[u] = __ldcs(reinterpret_cast<const float4*>(w + k));
                iv[u] = __ldcs(reinterpret_cast<const int4*>(idx + k));
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t k = k0 + 128 * u;
            if (k < e) {
                if (k >= b) acc[u] = fmaf(wv[u].x, gather<kShared>(x, iv[u].x), acc[u]);
                if (k + 1 >= b && k + 1 < e) acc[u] = fmaf(wv[u].y, gather<kShared>(x, iv[u].y), acc[u]);
                if (k + 2 >= b && k + 2 < e) acc[u] = fmaf(wv[u].z, gather<kShared>(x, iv[u].z), acc[u]);
                if (k + 3 >= b && k + 3 < e) acc[u] = fmaf(wv[u].w, gather<kShared>(x, iv[u].w), acc[u]);
            }
        }
    }
    return (acc[0] + acc[1]) + (acc[2] + acc[3]);
}

// lane_dot with 16-bit indices: four consecutive synapses' indices are one
// 8-byte load (little-endian halves); same blocks and summation order.
template <bool kShared>
__device__ __forceinline__ float lane_dot16(const float* w, const uint16_t* idx, const float* x, int64_t b,
                                            int64_t e, int lane) {
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (int64_t k0 = (b & ~int64_t(3)) + 4 * lane; k0 < e; k0 += 512) {
        float4 wv[4];
        uint2 iv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t k = k0 + 128 * u;
            if (k < e) {
                wv[u] = __ldcs(reinterpret_cast<const float4*>(w + k));
                iv[u] = __ldcs(reinterpret_cast<const uint2*>(idx + k));
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t k = k0 + 128 * u;
            if (k < e) {
                if (k >= b) acc[u] = fmaf(wv[u].x, gather<kShared>(x, (int32_t)(iv[u].x & 0xFFFFu)), acc[u]);
                if (k + 1 >= b && k + 1 < e) acc[u] = fmaf(wv[u].y, gather<kShared>(x, (int32_t)(iv[u].x >> 16)), acc[u]);
                if (k + 2 >= b && k + 2 < e) acc[u] = fmaf(wv[u].z, gather<kShared>(x, (int32_t)(iv[u].y & 0xFFFFu)), acc[u]);
                if (k + 3 >= b && k + 3 < e) acc[u] = fmaf(wv[u].w, gather<kShared>(x, (int32_t)(iv[u].y >> 16)), acc[u]);
            }
        }
    }
    return (acc[0] + acc[1]) + (acc[2] + acc[3]);
}

}  // namespace

// One warp per post neuron, or, for projections with short transposed rows,
// one lane per post (32 posts per work item).  kShared: the releases of the
// whole network (n_total floats) are first copied into shared memory, their
// whole 16-byte groups by asynchronous copies that every thread issues at
// once (a load-then-store loop would wait for each load in turn), the tail
// by plain loads.
template <bool kShared, bool kNarrow>
__global__ void __launch_bounds__(kShared ? kStagedThreads : kThreads, kShared ? 1 : 4) k_graded_spmv(const GradedArgs a) {
    extern __shared__ __align__(16) float s_x[];
    const float* x = a.r;
    if constexpr (kShared) {
        // (16-byte copies need a 16-byte aligned source; the release array is its own allocation)
        const int n4 = (reinterpret_cast<uintptr_t>(a.r) & 15u) == 0 ? a.n_total / 4 : 0;
        for (int i = threadIdx.x; i < n4; i += blockDim.x)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_u32(s_x + 4 * i)), "l"(a.r + 4 * i)
                         : "memory");
        for (int i = 4 * n4 + (int)threadIdx.x; i < a.n_total; i += blockDim.x) s_x[i] = a.r[i];
        asm volatile("cp.async.wait_all;" ::: "memory");
        __syncthreads();
        x = s_x;
    }
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t it = warp; it < a.spmv_items; it += warps) {
        int q = 0;
        while (a.gprojs[q].dense || a.gprojs[q].item_off + (a.gprojs[q].lane_rows ? (a.gprojs[q].n_post + 31) / 32
                                                                                  : a.gprojs[q].n_post) <= it)
            ++q;
        const GradProj& Q = a.gprojs[q];
        const float* xq = x + Q.pre_off;
        if (Q.lane_rows) {                           // 32 posts, one per lane, each row summed in order
            const int j = (int)(32 * (it - Q.item_off)) + lane;
            if (j < Q.n_post) {
                const int64_t jb = Q.csc_ptr[j], je = Q.csc_ptr[j + 1];
                float acc = 0.0f;
                for (int64_t k = jb; k < je; ++k) {
                    const int32_t i = kNarrow ? (int32_t)__ldg(Q.csc_pre16 + k) : __ldg(Q.csc_pre + k);
                    acc = fmaf(__ldg(Q.csc_w + k), gather<kShared>(xq, i), acc);
                }
                a.G[Q.g_off + j] = acc;
            }
            continue;
        }
        const int j = (int)(it - Q.item_off);
        float acc;
        if constexpr (kNarrow) acc = lane_dot16<kShared>(Q.csc_w, Q.csc_pre16, xq, Q.csc_ptr[j], Q.csc_ptr[j + 1], lane);
        else acc = lane_dot<kShared>(Q.csc_w, Q.csc_pre, xq, Q.csc_ptr[j], Q.csc_ptr[j + 1], lane);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) a.G[Q.g_off + j] = acc;
    }
}

__global__ void __launch_bounds__(kNeuronThreads) k_graded_neuron(const GradedArgs a) {
    const int idx_t = blockIdx.x * kNeuronThreads + threadIdx.x;     // tile-major over the SoA
    if (idx_t >= a.n_total) return;
    const int tile = idx_t / kTile;
    const int pop = a.tile_pop[tile];
    const DevPop& P = a.pops[pop];
    const int local = (tile - P.first_tile) * kTile + (idx_t % kTile);
    if (local >= P.n) return;
    const int idx = P.offset + local;
    float V = a.V[idx], m = a.m[idx], h = a.h[idx], n = a.n[idx], ie = a.iext[idx];
    if (P.thr_drive) {
        const uint4 r = philox_4x32_10(make_uint4((uint32_t)local, a.t_rng, P.tag, kStreamDrive),
                                       PhiloxKey{a.seed_lo, a.seed_hi});
        if (below(r.x, P.thr_drive)) ie += P.drive_amp;
    }
    if (a.rec_state) {                     // step-start state for the adjoint
        a.rec_state[idx] = V;
        a.rec_state[a.n_total + idx] = m;
        a.rec_state[2 * (size_t)a.n_total + idx] = h;
        a.rec_state[3 * (size_t)a.n_total + idx] = n;
        a.rec_state[4 * (size_t)a.n_total + idx] = ie;
        a.rec_r[idx] = a.r[idx];
    }
    float dI;
    const float isyn = graded_isyn(a, pop, local, V, &dI);
    const float I_in = isyn + ie;
    const HHCell cell{P.gNa, P.ENa, P.gK, P.EK, P.gL, P.EL};
    const float V0 = V;
    for (int s = 0; s < a.n_sub; ++s) hh_substep(cell, a.hs, P.hs_over_C, I_in, V, m, h, n);
    a.V[idx] = V; a.m[idx] = m; a.h[idx] = h; a.n[idx] = n;
    a.iext[idx] = ie * P.drive_dec;
    a.r[idx] = release(V, P.rel_thr, P.rel_inv_slope);
    if (V0 < P.v_thresh && V >= P.v_thresh) {
        atomicAdd(P.spike_count, 1ull);
        P.neuron_spikes[local] += 1;
    }
    if (isnan(V)) atomicAdd(P.nan_count, 1ull);
    if (pop == a.out_pop) {
        const float y = a.y[local] + a.a_filter * (V - a.y[local]);
        a.y[local] = y;
        if (a.y_out) a.y_out[(size_t)a.t_rec * a.n_out + local] = y;
    }
}

__global__ void k_graded_release_init(const GradedArgs a) {
    const int idx_t = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx_t >= a.n_total) return;
    const int tile = idx_t / kTile;
    const DevPop& P = a.pops[a.tile_pop[tile]];
    const int local = (tile - P.first_tile) * kTile + (idx_t % kTile);
    if (local >= P.n) return;
    a.r[P.offset + local] = release(a.V[P.offset + local], P.rel_thr, P.rel_inv_slope);
    if (a.tile_pop[tile] == a.out_pop) a.y[local] = a.V[P.offset + local];
}

// Reverse of one step for every neuron.  Reads the adjoint of the state after
// the step (lV includes the pre-synaptic gather of the later step), writes the
// local part of the adjoint of the state before it, dL/dG per incoming
// projection (per-step slice and time-contiguous copy) and dL/ds partials.
// kS: the substeps per step when known at compile time (the recomputed
// substep states then live in registers), 0 for the run-time count.
template <int kS>
__global__ void __launch_bounds__(kNeuronThreads) k_graded_reverse(const GradedArgs a, const AdjArgs b) {
    __shared__ double s_gs[kMaxGradedProjs];
    for (int k = threadIdx.x; k < a.n_gprojs; k += kNeuronThreads) s_gs[k] = 0.0;
    __syncthreads();
    // a warp's 32 neurons lie in one tile of one population (the SoA length
    // is a multiple of the tile), so pop is warp-uniform
    const int idx_t = blockIdx.x * kNeuronThreads + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int tile = idx_t / kTile;
    const int pop = a.tile_pop[tile];
    const DevPop& P = a.pops[pop];
    const int local = (tile - P.first_tile) * kTile + (idx_t % kTile);
    const bool active = local < P.n;
    const int idx = P.offset + local;
    float aI = 0.0f, V0 = 0.0f;
    if (active) {
        const size_t NT = (size_t)a.n_total;
        V0 = b.st[idx];
        const float m0 = b.st[NT + idx], h0 = b.st[2 * NT + idx], n0 = b.st[3 * NT + idx];
        const float ie = b.st[4 * NT + idx];
        float dIsyn_dV;
        const float isyn = graded_isyn(a, pop, local, V0, &dIsyn_dV);
        const float I_in = isyn + ie;
        const HHCell cell{P.gNa, P.ENa, P.gK, P.EK, P.gL, P.EL};
        // recompute the substep states (identical to the forward pass)
        constexpr int kCap = kS > 0 ? kS : kMaxSub;
        const int S = kS > 0 ? kS : a.n_sub;
        float Vs[kCap + 1], ms[kCap + 1], hs_[kCap + 1], ns[kCap + 1];
        Vs[0] = V0; ms[0] = m0; hs_[0] = h0; ns[0] = n0;
#pragma unroll
        for (int s = 0; s < kCap; ++s) {
            if (s < S) {
                float V = Vs[s], m = ms[s], h = hs_[s], n = ns[s];
                hh_substep(cell, a.hs, P.hs_over_C, I_in, V, m, h, n);
                Vs[s + 1] = V; ms[s + 1] = m; hs_[s + 1] = h; ns[s + 1] = n;
            }
        }
        float lV = b.lV[idx], lm = b.lm[idx], lh = b.lh[idx], ln = b.ln[idx];
        float ly_prev = 0.0f;
        if (pop == a.out_pop) {
            float ly = b.ly[local];
            ly += a.dL_dy[(size_t)a.t_rec * a.n_out + local];
            lV += a.a_filter * ly;
            ly_prev = (1.0f - a.a_filter) * ly;
        }
        const float c = P.hs_over_C;
#pragma unroll
        for (int s = kCap - 1; s >= 0; --s) {
            if (s < S) {
                const float V = Vs[s], m = ms[s], h = hs_[s], n = ns[s];
                const HHRates r = hh_rates(V);
                const HHDerivs d = hh_rate_derivs(V, r);
                const float m2 = m * m, m3 = m2 * m, n3 = n * n * n;
                const float dI_dV = P.gNa * m3 * h + P.gK * n3 * n + P.gL;
                const float dI_dm = 3.0f * P.gNa * m2 * h * (V - P.ENa);
                const float dI_dh = P.gNa * m3 * (V - P.ENa);
                const float dI_dn = 4.0f * P.gK * n3 * (V - P.EK);
                const float nV = lV * (1.0f - c * dI_dV) + lm * a.hs * (d.am * (1.0f - m) - d.bm * m) +
                                 lh * a.hs * (d.ah * (1.0f - h) - d.bh * h) + ln * a.hs * (d.an * (1.0f - n) - d.bn * n);
                const float nm = lV * (-c * dI_dm) + lm * (1.0f - a.hs * (r.am + r.bm));
                const float nh = lV * (-c * dI_dh) + lh * (1.0f - a.hs * (r.ah + r.bh));
                const float nn = lV * (-c * dI_dn) + ln * (1.0f - a.hs * (r.an + r.bn));
                aI = fmaf(lV, c, aI);
                lV = nV; lm = nm; lh = nh; ln = nn;
            }
        }
        b.lV_loc[idx] = fmaf(aI, dIsyn_dV, lV);
        b.lm[idx] = lm; b.lh[idx] = lh; b.ln[idx] = ln;
        if (pop == a.out_pop) b.ly[local] = ly_prev;
    }
    // dL/dG of the step and the scale gradients: the warp sums its neurons'
    // contributions before one shared atomic per projection
    const int qb = a.in_begin[pop], qe = a.in_begin[pop + 1];
    for (int k = qb; k < qe; ++k) {
        const int qi = a.in_list[k];
        const GradProj& q = a.gprojs[qi];
        double gs = 0.0;
        if (active) {
            const float nu = aI * q.scale * (q.E - V0);
            b.nu_step[q.g_off + local] = nu;
            b.nu_km[(size_t)(q.g_off + local) * b.kp + b.tl] = nu;
            gs = (double)aI * (double)(q.E - V0) * (double)a.G[q.g_off + local];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) gs += __shfl_xor_sync(0xffffffffu, gs, o);
        if (lane == 0 && gs != 0.0) atomicAdd(&s_gs[qi], gs);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < a.n_gprojs; k += kNeuronThreads)
        if (s_gs[k] != 0.0) atomicAdd(b.grad_scale + k, s_gs[k]);
}

// dL/dV_i = local part + r'_i sum over outgoing rows of w * dL/dG (one warp per neuron).
// One warp per pre-synaptic neuron; the dL/dG vector is gathered through L1
// (it fits there, and a shared-memory copy would take the L1's space).
// kShared: dL/dG of the step (total_posts floats) is first copied into shared
// memory, as the forward product stages the releases, so the rows' random
// reads of it cost bank conflicts instead of L1 / L2 round trips.
template <bool kShared>
__global__ void __launch_bounds__(kShared ? kStagedThreads : kThreads, kShared ? 1 : 4) k_graded_gather(const GradedArgs a,
                                                                                                         const AdjArgs b) {
    extern __shared__ __align__(16) float s_nu[];
    const float* nu_all = b.nu_step;
    if constexpr (kShared) {
        const int n = (int)a.total_posts;
        const int n4 = (reinterpret_cast<uintptr_t>(b.nu_step) & 15u) == 0 ? n / 4 : 0;
        for (int i = threadIdx.x; i < n4; i += blockDim.x)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_u32(s_nu + 4 * i)),
                         "l"(b.nu_step + 4 * i) : "memory");
        for (int i = 4 * n4 + (int)threadIdx.x; i < n; i += blockDim.x) s_nu[i] = b.nu_step[i];
        asm volatile("cp.async.wait_all;" ::: "memory");
        __syncthreads();
        nu_all = s_nu;
    }
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t w = warp; w < a.n_total; w += warps) {
        const int tile = (int)(w / kTile);
        const int pop = a.tile_pop[tile];
        const DevPop& P = a.pops[pop];
        const int local = (tile - P.first_tile) * kTile + (int)(w % kTile);
        if (local >= P.n) continue;
        const int idx = P.offset + local;
        float acc = 0.0f;
        for (int k = a.out_begin[pop]; k < a.out_begin[pop + 1]; ++k) {
            const GradProj& q = a.gprojs[a.out_list[k]];
            const float* nu = nu_all + q.g_off;
            if (q.dense) {
                // the neuron's row of the matrix against dL/dG of all posts
                const float* row = q.w + (int64_t)local * q.n_post;
                if ((q.n_post & 3) == 0 && (q.g_off & 3) == 0) {
#pragma unroll 4
                    for (int j = 4 * lane; j < q.n_post; j += 128) {
                        const float4 w4 = __ldg(reinterpret_cast<const float4*>(row + j));   // may stay in L2
                        const float4 v4 = *reinterpret_cast<const float4*>(nu + j);
                        acc = fmaf(w4.x, v4.x, acc);
                        acc = fmaf(w4.y, v4.y, acc);
                        acc = fmaf(w4.z, v4.z, acc);
                        acc = fmaf(w4.w, v4.w, acc);
                    }
                } else {
                    for (int j = lane; j < q.n_post; j += 32) acc = fmaf(row[j], nu[j], acc);
                }
                continue;
            }
            const int64_t rb = q.row_ptr[local], re = q.row_ptr[local + 1];
            if (kShared && q.col16) {
                // 16-byte weight and 8-byte index loads of 4 synapses per lane,
                // four 128-synapse blocks in flight, dL/dG from shared memory
                acc += lane_dot16<true>(q.w, q.col16, nu, rb, re, lane);
            } else if (q.col16) {
                for (int64_t e = rb + lane; e < re; e += 32) acc = fmaf(q.w[e], nu[q.col16[e]], acc);
            } else {
                for (int64_t e = rb + lane; e < re; e += 32) acc = fmaf(q.w[e], nu[q.col[e]], acc);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            const float r = b.r_step[idx];
            b.lV[idx] = fmaf(r * (1.0f - r) * P.rel_inv_slope, acc, b.lV_loc[idx]);
        }
    }
}

// dL/dw_ik += sum over the segment's steps of r_i(t) dL/dG_q[k](t); one warp
// per compressed row, the row's releases staged in shared memory.
__global__ void __launch_bounds__(kThreads) k_graded_sddmm(const GradedArgs a, const AdjArgs b, int qi,
                                                           float* grad_w, int L) {
    __shared__ float s_r[kThreads / 32][kMaxSeg];
    const GradProj& q = a.gprojs[qi];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t warps = (int64_t)gridDim.x * (kThreads / 32);
    const size_t NT = (size_t)a.n_total;
    for (int64_t i = (int64_t)blockIdx.x * (kThreads / 32) + wib; i < q.n_pre; i += warps) {
        for (int t = lane; t < L; t += 32) s_r[wib][t] = b.r_seg[(size_t)t * NT + q.pre_off + i];
        __syncwarp();
        for (int64_t e = q.row_ptr[i] + lane; e < q.row_ptr[i + 1]; e += 32) {
            const float* nu = b.nu_km + (size_t)(q.g_off + q.col[e]) * b.kp;
            float acc = 0.0f;
            int t = 0;
            for (; t + 4 <= L; t += 4) {
                const float4 v = *reinterpret_cast<const float4*>(nu + t);
                acc = fmaf(s_r[wib][t], v.x, acc);
                acc = fmaf(s_r[wib][t + 1], v.y, acc);
                acc = fmaf(s_r[wib][t + 2], v.z, acc);
                acc = fmaf(s_r[wib][t + 3], v.w, acc);
            }
            for (; t < L; ++t) acc = fmaf(s_r[wib][t], nu[t], acc);
            grad_w[e] += acc;
        }
        __syncwarp();
    }
}

__global__ void k_scatter_csc(const float* w_csr, const int64_t* perm, float* w_csc, int64_t nnz) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
        w_csc[e] = w_csr[perm[e]];
}

__global__ void k_finish_grad_scale(const double* acc, const float* scale_of, float* out, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) out[k] = (float)acc[k];
    (void)scale_of;
}

// ---- launchers ---------------------------------------------------------------
static int grid_warps(int64_t warps) {
    int64_t b = (warps + (kThreads / 32) - 1) / (kThreads / 32);
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (int)b;
}

// Staged launch: one 1024-thread CTA per SM with `bytes` of shared memory.
template <typename K, typename... Args>
static cudaError_t launch_staged(K kernel, size_t bytes, cudaStream_t s, Args... args) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    kernel<<<sms, kStagedThreads, bytes, s>>>(args...);
    return cudaGetLastError();
}

cudaError_t launch_graded_spmv(const GradedArgs& a, cudaStream_t s) {
    if (a.spmv_items == 0) return cudaSuccess;
    const size_t bytes = sizeof(float) * (size_t)a.n_total;
    if (bytes <= kStageMaxBytes)
        return a.narrow ? launch_staged(k_graded_spmv<true, true>, bytes, s, a)
                        : launch_staged(k_graded_spmv<true, false>, bytes, s, a);
    if (a.narrow) k_graded_spmv<false, true><<<grid_warps(a.spmv_items), kThreads, 0, s>>>(a);
    else k_graded_spmv<false, false><<<grid_warps(a.spmv_items), kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_graded_neuron(const GradedArgs& a, cudaStream_t s) {
    k_graded_neuron<<<(a.n_total + kNeuronThreads - 1) / kNeuronThreads, kNeuronThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_graded_release_init(const GradedArgs& a, cudaStream_t s) {
    k_graded_release_init<<<(a.n_total + kThreads - 1) / kThreads, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_graded_reverse(const GradedArgs& a, const AdjArgs& b, cudaStream_t s) {
    const int grid = (a.n_total + kNeuronThreads - 1) / kNeuronThreads;
    if (a.n_sub == 4) k_graded_reverse<4><<<grid, kNeuronThreads, 0, s>>>(a, b);
    else k_graded_reverse<0><<<grid, kNeuronThreads, 0, s>>>(a, b);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t bytes = sizeof(float) * (size_t)a.total_posts;
    if (bytes <= kStageMaxBytes) return launch_staged(k_graded_gather<true>, bytes, s, a, b);
    k_graded_gather<false><<<grid_warps(a.n_total), kThreads, 0, s>>>(a, b);
    return cudaGetLastError();
}

cudaError_t launch_graded_sddmm(const GradedArgs& a, const AdjArgs& b, int q, int64_t n_pre, float* grad_w, int L,
                                cudaStream_t s) {
    if (n_pre == 0 || L == 0) return cudaSuccess;
    k_graded_sddmm<<<grid_warps(n_pre), kThreads, 0, s>>>(a, b, q, grad_w, L);
    return cudaGetLastError();
}

cudaError_t launch_scatter_csc(const float* w_csr, const int64_t* perm, float* w_csc, int64_t nnz, cudaStream_t s) {
    if (nnz == 0) return cudaSuccess;
    const int blocks = (int)std::min<int64_t>((nnz + 255) / 256, 4096);
    k_scatter_csc<<<blocks, 256, 0, s>>>(w_csr, perm, w_csc, nnz);
    return cudaGetLastError();
}

cudaError_t launch_finish_grad_scale(const double* acc, float* out, int n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_finish_grad_scale<<<1, 256, 0, s>>>(acc, nullptr, out, n);
    return cudaGetLastError();
}

}  // namespace snn
