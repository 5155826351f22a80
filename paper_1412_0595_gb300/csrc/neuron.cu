// Fused per-neuron step kernel (Sec. 2: HH neurons advanced at discrete time
// steps) with ordered spike compaction.
//
// One CTA handles one tile of kTile neurons of one population, one neuron per
// thread, state in structure-of-arrays FP32 (coalesced 128 B per warp per
// array).  Tiles take a ticket from a monotone counter, so tile k of a step
// always starts after tile k-1 of the same step has a ticket; the ticket also
// gives the step epoch (ticket / num_tiles), which drives the counter-based
// random numbers and tags the tile status words, so nothing is reset between
// steps.  The ascending spike list is built with a warp ballot, a CTA scan
// and a decoupled look-back over the preceding tiles of the population; every
// look-back wait is bounded and reports SNN_ERR_TIMEOUT through the sticky
// error word instead of hanging.
#include "device_math.cuh"
#include "snn_internal.cuh"

namespace snn {

namespace {

__device__ __forceinline__ unsigned long long wait_tile(const unsigned long long* p, uint32_t epoch,
                                                        uint32_t limit, uint32_t* err) {
    for (uint32_t it = 0;; ++it) {
        const unsigned long long s = ld_acquire_u64(p);
        if ((uint32_t)(s >> 32) == epoch && (s & (kFlagAgg | kFlagPrefix))) return s;
        if (it >= limit) {
            atomicOr(err, kDevErrTimeout);
            return ((unsigned long long)epoch << 32) | kFlagPrefix;   // give up: count 0
        }
        if (it > 64) __nanosleep(64);
    }
}

// Exclusive prefix of this tile's spike count within its population, by
// decoupled look-back (executed by warp 0; returns the value in all lanes).
__device__ __forceinline__ int tile_prefix(const NeuronArgs& a, int tile, int first_tile,
                                           uint32_t epoch, int total) {
    const int lane = threadIdx.x & 31;
    unsigned long long* status = a.tile_status;
    const unsigned long long tagged = (unsigned long long)epoch << 32;
    if (tile == first_tile) {
        if (lane == 0) st_release_u64(status + tile, tagged | kFlagPrefix | (unsigned long long)total);
        return 0;
    }
    if (lane == 0) st_release_u64(status + tile, tagged | kFlagAgg | (unsigned long long)total);
    int excl = 0;
    int k = tile - 1;
    while (true) {
        const int idx = k - lane;
        unsigned long long s;
        if (idx >= first_tile) s = wait_tile(status + idx, epoch, a.spin_limit, a.error);
        else s = tagged | kFlagPrefix;          // before the population: prefix 0
        const bool is_prefix = (s & kFlagPrefix) != 0;
        const int val = (int)(s & kCountMask);
        const unsigned pm = __ballot_sync(0xffffffffu, is_prefix);
        if (pm) {
            const int stop = __ffs(pm) - 1;     // nearest predecessor with a full prefix
            int v = lane <= stop ? val : 0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            excl += v;
            break;
        }
        int v = val;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        excl += v;
        k -= 32;
    }
    if (lane == 0) st_release_u64(status + tile, tagged | kFlagPrefix | (unsigned long long)(excl + total));
    return excl;
}

__device__ __forceinline__ int find_pop(const int32_t* tile_pop, int tile) { return tile_pop[tile]; }

}  // namespace

__global__ void __launch_bounds__(kTile) k_neuron_step(const NeuronArgs a) {
    __shared__ unsigned long long s_ticket;
    __shared__ int s_warp[kTile / 32];
    __shared__ int s_base;
    if (threadIdx.x == 0) s_ticket = atomicAdd(a.ticket, 1ull);
    __syncthreads();
    const unsigned long long ticket = s_ticket;
    const int tile = (int)(ticket % (unsigned long long)a.num_tiles);
    const unsigned long long epoch64 = ticket / (unsigned long long)a.num_tiles;
    const uint32_t epoch = (uint32_t)epoch64;
    const uint32_t t = (uint32_t)(epoch64 - *a.epoch_base);      // simulated step
    const int p = find_pop(a.tile_pop, tile);
    const DevPop& P = a.pops[p];
    const int local = (tile - P.first_tile) * kTile + (int)threadIdx.x;
    const bool active = local < P.n;
    const int idx = P.offset + local;
    const PhiloxKey key{a.seed_lo, a.seed_hi};

    bool spike = false;
    bool is_nan = false;
    if (active) {
        if (P.kind == SNN_POP_SOURCE) {
            const uint4 r = philox_4x32_10(make_uint4((uint32_t)local, t, P.tag, kStreamSource), key);
            spike = below(r.x, P.thr_src);
        } else {
            float V = a.V[idx], m = a.m[idx], h = a.h[idx], n = a.n[idx];
            float g0 = a.g0[idx], g1 = a.g1[idx], ie = a.iext[idx];
            if (P.thr_drive) {
                const uint4 r = philox_4x32_10(make_uint4((uint32_t)local, t, P.tag, kStreamDrive), key);
                if (below(r.x, P.thr_drive)) ie += P.drive_amp;
            }
            const float isyn = g0 * (P.E0 - V) + g1 * (P.E1 - V);
            const float I_in = isyn + ie;
            const HHCell cell{P.gNa, P.ENa, P.gK, P.EK, P.gL, P.EL};
            float v = V;
            for (int s = 0; s < a.n_sub; ++s) hh_substep(cell, a.hs, P.hs_over_C, I_in, v, m, h, n);
            spike = (V < P.v_thresh) && (v >= P.v_thresh);
            is_nan = isnan(v);
            a.V[idx] = v;
            a.m[idx] = m;
            a.h[idx] = h;
            a.n[idx] = n;
            a.g0[idx] = g0 * P.d0;
            a.g1[idx] = g1 * P.d1;
            a.iext[idx] = ie * P.drive_dec;
            if (a.isyn_rec) a.isyn_rec[idx] = isyn;
        }
    }

    // ---- ordered compaction ------------------------------------------------
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned ballot = __ballot_sync(0xffffffffu, spike);
    const unsigned nan_ballot = __ballot_sync(0xffffffffu, is_nan);
    if (lane == 0) {
        s_warp[warp] = __popc(ballot);
        if (nan_ballot) atomicAdd(P.nan_count, (unsigned long long)__popc(nan_ballot));
    }
    __syncthreads();
    if (warp == 0) {
        const int c = lane < kTile / 32 ? s_warp[lane] : 0;
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        const int excl = tile_prefix(a, tile, P.first_tile, epoch, total);
        if (lane < kTile / 32) s_warp[lane] = incl - c;
        if (lane == 0) {
            s_base = excl;
            if (tile == P.first_tile + P.n_tiles - 1) *P.nspk = excl + total;
            if (total) atomicAdd(P.spike_count, (unsigned long long)total);
        }
    }
    __syncthreads();
    if (spike) {
        const unsigned lower = ballot & ((1u << lane) - 1u);
        P.spk[s_base + s_warp[warp] + __popc(lower)] = local;
        P.neuron_spikes[local] += 1;
    }
}

__global__ void k_init_state(const DevPop* pops, const int32_t* tile_pop, float* V, float* m,
                             float* h, float* n, float* g0, float* g1, float* iext) {
    const int tile = blockIdx.x;
    const DevPop& P = pops[tile_pop[tile]];
    const int local = (tile - P.first_tile) * kTile + (int)threadIdx.x;
    const int idx = P.offset + local;
    float v = V[idx], mm = 0.f, hh = 0.f, nn = 0.f;
    if (local < P.n && P.kind == SNN_POP_HH) hh_steady(v, mm, hh, nn);
    m[idx] = mm;
    h[idx] = hh;
    n[idx] = nn;
    g0[idx] = 0.f;
    g1[idx] = 0.f;
    iext[idx] = 0.f;
}

__global__ void k_set_epoch_base(unsigned long long* ticket, int num_tiles) {
    ticket[1] = ticket[0] / (unsigned long long)num_tiles;
}

cudaError_t launch_neuron_step(const NeuronArgs& a, cudaStream_t s) {
    if (a.num_tiles == 0) return cudaSuccess;
    k_neuron_step<<<a.num_tiles, kTile, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_init_state(const DevPop* pops, int, const int32_t* tile_pop, int num_tiles,
                              float* V, float* m, float* h, float* n, float* g0, float* g1,
                              float* iext, cudaStream_t s) {
    if (num_tiles == 0) return cudaSuccess;
    k_init_state<<<num_tiles, kTile, 0, s>>>(pops, tile_pop, V, m, h, n, g0, g1, iext);
    return cudaGetLastError();
}

cudaError_t launch_set_epoch_base(unsigned long long* ticket, int num_tiles, cudaStream_t s) {
    k_set_epoch_base<<<1, 1, 0, s>>>(ticket, num_tiles > 0 ? num_tiles : 1);
    return cudaGetLastError();
}

}  // namespace snn
