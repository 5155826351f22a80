// Persistent step engine: one cooperative launch advances the network by many
// time steps, with a single grid-wide barrier per step.
//
// Small networks spend most of a two-kernel step in launch latency, so here
// every CTA stays resident and loops over the steps.  Each tile updates its
// neurons (the same per-neuron code as the plain engine), then pushes the rows
// of its own spiking neurons into a double-buffered event accumulator: the
// events of step e land in buffer e & 1, and the owner of a post neuron folds
// buffer (e - 1) & 1 into its conductance at the start of step e and clears
// it.  The one-step delay of the model is therefore kept without a separate
// propagation phase, and one barrier per step separates producers from
// consumers.  Spike lists, list lengths and counters are kept exactly as in
// the plain engine, so the two engines can alternate.  When the
// grid holds one CTA per tile, each thread keeps its neuron's state in
// registers for the whole launch.  The barrier wait is bounded and reports
// SNN_ERR_TIMEOUT; after a timeout every CTA leaves the kernel.
#include "compaction.cuh"
#include "neuron_update.cuh"

namespace snn {

namespace {

// Grid-wide barrier on a monotone counter: arrive with one atomic after a
// fence, then poll until every CTA of this barrier has arrived.  Returns false
// when the wait ran out (the error word then holds SNN_ERR_TIMEOUT and the
// caller leaves the kernel; the other CTAs run out of their own waits).
__device__ __forceinline__ bool grid_sync(GridBarrier* b, unsigned long long target, uint32_t limit,
                                          uint32_t* err) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        atomicAdd(&b->count, 1ull);
        for (uint32_t it = 0; ld_acquire_u64(&b->count) < target; ++it) {
            if (it >= limit) {
                atomicOr(err, kDevErrTimeout);
                ok = 0;
                break;
            }
            if (it > 16) __nanosleep(20);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Adds scale * w of row i of projection q into buffer `buf` of its accumulator.
// Called by the push warps (threads 32 .. kTile-1) of the CTA.
__device__ __forceinline__ void push_row(const DevProj& q, int i, float* dst, int pt, int npt) {
    const float s = q.scale;
    if (q.layout == SNN_LAYOUT_CSR) {
        const int64_t beg = q.row_ptr[i], end = q.row_ptr[i + 1];
        for (int64_t k = (beg & ~int64_t(3)) + 4 * (int64_t)pt; k < end; k += 4 * (int64_t)npt) {
            const int4 c4 = __ldg(reinterpret_cast<const int4*>(q.col + k));
            const float4 w4 = __ldg(reinterpret_cast<const float4*>(q.w + k));
            if (k >= beg) atomicAdd(dst + c4.x, s * w4.x);
            if (k + 1 >= beg && k + 1 < end) atomicAdd(dst + c4.y, s * w4.y);
            if (k + 2 >= beg && k + 2 < end) atomicAdd(dst + c4.z, s * w4.z);
            if (k + 3 >= beg && k + 3 < end) atomicAdd(dst + c4.w, s * w4.w);
        }
    } else {
        const int n_post = q.n_post;
        const float* row = q.w + (int64_t)i * n_post;
        if ((n_post & 3) == 0) {
            for (int j = 4 * pt; j < n_post; j += 4 * npt) {
                const float4 w4 = __ldg(reinterpret_cast<const float4*>(row + j));
                atomicAdd(reinterpret_cast<float4*>(dst + j), make_float4(s * w4.x, s * w4.y, s * w4.z, s * w4.w));
            }
        } else {
            for (int j = pt; j < n_post; j += npt) atomicAdd(dst + j, s * __ldg(row + j));
        }
    }
}

template <bool kResident>
__global__ void __launch_bounds__(kTile, 6) k_step_persistent(const PersistArgs A) {
    __shared__ int s_off[kTile / 32];
    __shared__ int s_spk[kTile];
    __shared__ int s_total, s_base;
    __shared__ DevPop s_pop;
    const NeuronArgs& a = A.n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned long long T0 = *a.ticket;                 // a multiple of num_tiles
    const unsigned long long epoch0 = T0 / (unsigned long long)a.num_tiles;
    const unsigned long long ebase = *a.epoch_base;
    const PhiloxKey key{a.seed_lo, a.seed_hi};
    const int NT = A.acc_stride;
    const unsigned long long bar_base = A.bar->base;

    // resident mode: this CTA's single tile and its neuron's state
    NeuronState rs{};
    const int my_tile = blockIdx.x;
    if (kResident && my_tile < a.num_tiles) {
        const DevPop& P = a.pops[a.tile_pop[my_tile]];
        const int local = (my_tile - P.first_tile) * kTile + (int)threadIdx.x;
        const int idx = P.offset + local;
        if (local < P.n && P.kind != SNN_POP_SOURCE)
            rs = NeuronState{a.V[idx], a.m[idx], a.h[idx], a.n[idx], a.g0[idx], a.g1[idx], a.iext[idx]};
    }

    for (int k = 0; k < A.n_steps; ++k) {
        const unsigned long long e64 = epoch0 + (unsigned long long)k;
        const uint32_t t = (uint32_t)(e64 - ebase);
        const int slot = (int)(e64 & 1ull);
        const int prev = (int)((e64 + 1ull) & 1ull) * NT;    // buffer of step e - 1
        const int cur = (int)(e64 & 1ull) * NT;              // buffer of step e
        for (int tile = blockIdx.x; tile < a.num_tiles; tile += gridDim.x) {
            if (!kResident || k == 0) {
                __syncthreads();                      // previous readers of s_pop are done
                copy_pop(&s_pop, a.pops + a.tile_pop[tile]);
                __syncthreads();
            }
            const DevPop& P = s_pop;
            const int local = (tile - P.first_tile) * kTile + (int)threadIdx.x;
            const bool active = local < P.n;
            const int idx = P.offset + local;
            bool spike = false, is_nan = false;
            if (active) {
                NeuronState s{};
                if (P.kind != SNN_POP_SOURCE) {
                    if (kResident) s = rs;
                    else s = NeuronState{a.V[idx], a.m[idx], a.h[idx], a.n[idx], __ldcg(a.g0 + idx),
                                         __ldcg(a.g1 + idx), a.iext[idx]};
                    // events of the previous step, delivered by any CTA
                    const float in0 = __ldcg(A.acc0 + prev + idx);
                    const float in1 = __ldcg(A.acc1 + prev + idx);
                    if (in0 != 0.0f) { s.g0 += in0; __stcg(A.acc0 + prev + idx, 0.0f); }
                    if (in1 != 0.0f) { s.g1 += in1; __stcg(A.acc1 + prev + idx, 0.0f); }
                }
                float isyn;
                spike = neuron_step(P, key, t, local, a.hs, a.n_sub, s, &isyn);
                if (P.kind != SNN_POP_SOURCE) {
                    is_nan = isnan(s.V);
                    if (kResident) {
                        rs = s;
                    } else {
                        a.V[idx] = s.V; a.m[idx] = s.m; a.h[idx] = s.h; a.n[idx] = s.n;
                        __stcg(a.g0 + idx, s.g0); __stcg(a.g1 + idx, s.g1); a.iext[idx] = s.ie;
                    }
                    if (a.isyn_rec) a.isyn_rec[idx] = isyn;
                }
            }
            if (tile == P.first_tile && threadIdx.x == 0) P.nspk[slot ^ 1] = 0;   // next step's count
            const unsigned ballot = __ballot_sync(0xffffffffu, spike);
            const unsigned nan_ballot = __ballot_sync(0xffffffffu, is_nan);
            if (lane == 0 && nan_ballot) atomicAdd(P.nan_count, (unsigned long long)__popc(nan_ballot));
            const int total = tile_claim(spike, ballot, s_off, &s_total, &s_base, P.nspk + slot);
            if (spike) {
                const int r = s_off[warp] + __popc(ballot & ((1u << lane) - 1u));
                s_spk[r] = local;
                P.spk[s_base + r] = local;
                P.neuron_spikes[local] += 1;
            }
            if (total) {
                if (threadIdx.x == 0) atomicAdd(P.spike_count, (unsigned long long)total);
                __syncthreads();
                // push the rows of this tile's spikes into buffer `cur`
                const int pop = a.tile_pop[tile];
                const int qb = A.out_begin[pop], qe = A.out_begin[pop + 1];
                for (int sidx = 0; sidx < total; ++sidx) {
                    const int i = s_spk[sidx];
                    for (int qq = qb; qq < qe; ++qq) {
                        const DevProj& Q = A.projs[A.out_list[qq]];
                        push_row(Q, i, Q.acc + cur, threadIdx.x, kTile);
                    }
                }
                __syncthreads();
            }
        }
        if (!grid_sync(A.bar, bar_base + (unsigned long long)(k + 1) * gridDim.x + (unsigned long long)A.barrier_extra,
                       a.spin_limit, a.error))
            return;
    }

    // fold the last step's events into the conductances and clear the buffer
    const unsigned long long e_last = epoch0 + (unsigned long long)A.n_steps - 1ull;
    const int last = (int)(e_last & 1ull) * NT;
    for (int tile = blockIdx.x; tile < a.num_tiles; tile += gridDim.x) {
        const DevPop& P = a.pops[a.tile_pop[tile]];
        const int local = (tile - P.first_tile) * kTile + (int)threadIdx.x;
        if (local >= P.n || P.kind == SNN_POP_SOURCE) continue;
        const int idx = P.offset + local;
        NeuronState s = rs;
        if (!kResident) s.g0 = __ldcg(a.g0 + idx), s.g1 = __ldcg(a.g1 + idx);
        if (A.n_steps > 0) {
            const float in0 = __ldcg(A.acc0 + last + idx), in1 = __ldcg(A.acc1 + last + idx);
            s.g0 += in0;
            s.g1 += in1;
            __stcg(A.acc0 + last + idx, 0.0f);
            __stcg(A.acc1 + last + idx, 0.0f);
        }
        if (kResident) {
            a.V[idx] = s.V; a.m[idx] = s.m; a.h[idx] = s.h; a.n[idx] = s.n; a.iext[idx] = s.ie;
        }
        a.g0[idx] = s.g0;
        a.g1[idx] = s.g1;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *a.ticket = T0 + (unsigned long long)A.n_steps * (unsigned long long)a.num_tiles;
        A.bar->base = bar_base + (unsigned long long)A.n_steps * gridDim.x;
    }
}

}  // namespace

cudaError_t persistent_capacity(int sm_count, int* blocks) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_persistent<false>, kTile, 0);
    if (e != cudaSuccess) return e;
    int per_sm_r = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_r, k_step_persistent<true>, kTile, 0);
    if (e != cudaSuccess) return e;
    *blocks = sm_count * std::min(per_sm, per_sm_r);
    return cudaSuccess;
}

cudaError_t launch_persistent(const PersistArgs& a, int grid, cudaStream_t s) {
    if (a.n.num_tiles == 0 || a.n_steps <= 0) return cudaSuccess;
    void* args[] = {const_cast<PersistArgs*>(&a)};
    if (grid >= a.n.num_tiles)
        return cudaLaunchCooperativeKernel((const void*)k_step_persistent<true>, dim3(a.n.num_tiles), dim3(kTile),
                                           args, 0, s);
    return cudaLaunchCooperativeKernel((const void*)k_step_persistent<false>, dim3(grid), dim3(kTile), args, 0, s);
}

}  // namespace snn
