// Fused per-neuron step kernel (Sec. 2: HH neurons advanced at discrete time
// steps) with spike compaction, for the two-kernel step of the plain engine.
//
// One CTA handles one tile of kTile neurons of one population, two neighbour
// neurons per thread, state in structure-of-arrays FP32 (coalesced 256 B per
// warp per array).  Tiles take a ticket from a monotone counter; the ticket gives the
// step epoch (ticket / num_tiles), which drives the counter-based random
// numbers and the parity of the double-buffered list lengths, so nothing is
// reset between steps and no tile waits for another.
#include <algorithm>

#include "compaction.cuh"
#include "neuron_update.cuh"

namespace snn {

// One CTA of kTile / 2 threads per tile; thread t holds the tile's neurons
// 2 t and 2 t + 1 (8-byte loads and stores of each state array) and steps
// them together (FP32x2 arithmetic for HH populations).  Channel 1 and the
// drive current are read and written only for populations where they can be
// nonzero.
__global__ void __launch_bounds__(kTile / 2, 6) k_neuron_step(const NeuronArgs a) {
    __shared__ int s_off[kTile / 64];
    __shared__ int s_total, s_base;
    __shared__ uint32_t s_t;
    __shared__ int s_slot;
    __shared__ DevPop s_pop;
    // This CTA's tiles are blockIdx.x, blockIdx.x + gridDim.x, ...  It takes
    // that many tickets with one atomic add; whatever the order of the CTAs,
    // every ticket of one launch lies in [e * num_tiles, (e + 1) * num_tiles),
    // so ticket / num_tiles is the step epoch e.
    const int my_tiles = (a.num_tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
    if (threadIdx.x == 0) {
        const unsigned long long ticket = atomicAdd(a.ticket, (unsigned long long)my_tiles);
        const unsigned long long epoch = ticket / (unsigned long long)a.num_tiles;
        s_t = (uint32_t)(epoch - *a.epoch_base);          // simulated step
        s_slot = (int)(epoch & 1ull);
    }
    __syncthreads();
    const uint32_t t = s_t;
    const int slot = s_slot;
    const PhiloxKey key{a.seed_lo, a.seed_hi};
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int cur_pop = -1;
    for (int tile = blockIdx.x; tile < a.num_tiles; tile += gridDim.x) {
        const int p = a.tile_pop[tile];
        if (p != cur_pop) {                                  // uniform: a new population descriptor
            __syncthreads();
            copy_pop(&s_pop, a.pops + p);
            __syncthreads();
            cur_pop = p;
        }
        const DevPop& P = s_pop;
        const int local = (tile - P.first_tile) * kTile + 2 * (int)threadIdx.x;
        const unsigned live = (local < P.n ? 1u : 0u) | (local + 1 < P.n ? 2u : 0u);
        const int idx = P.offset + local;                    // even: 8-byte aligned pairs
        if (tile == P.first_tile && threadIdx.x == 0) P.nspk[slot ^ 1] = 0;   // next step's count

        unsigned spike = 0u, is_nan = 0u;
        if (live) {
            NeuronPair s{};
            const bool hh_like = P.kind != SNN_POP_SOURCE;
            if (hh_like) {
                s.V = *reinterpret_cast<const float2*>(a.V + idx);
                s.m = *reinterpret_cast<const float2*>(a.m + idx);
                s.h = *reinterpret_cast<const float2*>(a.h + idx);
                s.n = *reinterpret_cast<const float2*>(a.n + idx);
                s.g0 = *reinterpret_cast<const float2*>(a.g0 + idx);
                if (P.g1_live) s.g1 = *reinterpret_cast<const float2*>(a.g1 + idx);
                if (P.iext_live) s.ie = *reinterpret_cast<const float2*>(a.iext + idx);
            }
            float2 isyn;
            spike = neuron_step_pair(P, key, t, local, a.hs, a.n_sub, s, &isyn) & live;
            if (hh_like) {
                is_nan = (isnan(s.V.x) ? 1u : 0u) | (isnan(s.V.y) ? 2u : 0u);
                is_nan &= live;
                if (live == 3u) {
                    *reinterpret_cast<float2*>(a.V + idx) = s.V;
                    *reinterpret_cast<float2*>(a.m + idx) = s.m;
                    *reinterpret_cast<float2*>(a.h + idx) = s.h;
                    *reinterpret_cast<float2*>(a.n + idx) = s.n;
                    *reinterpret_cast<float2*>(a.g0 + idx) = s.g0;
                    if (P.g1_live) *reinterpret_cast<float2*>(a.g1 + idx) = s.g1;
                    if (P.iext_live) *reinterpret_cast<float2*>(a.iext + idx) = s.ie;
                    if (a.isyn_rec) *reinterpret_cast<float2*>(a.isyn_rec + idx) = isyn;
                } else {                                     // the second half is a padding slot
                    a.V[idx] = s.V.x; a.m[idx] = s.m.x; a.h[idx] = s.h.x; a.n[idx] = s.n.x;
                    a.g0[idx] = s.g0.x;
                    if (P.g1_live) a.g1[idx] = s.g1.x;
                    if (P.iext_live) a.iext[idx] = s.ie.x;
                    if (a.isyn_rec) a.isyn_rec[idx] = isyn.x;
                }
            }
        }

        const unsigned b0 = __ballot_sync(0xffffffffu, spike & 1u);
        const unsigned b1 = __ballot_sync(0xffffffffu, spike & 2u);
        const int nans = __popc(__ballot_sync(0xffffffffu, is_nan & 1u)) + __popc(__ballot_sync(0xffffffffu, is_nan & 2u));
        if (lane == 0 && nans) atomicAdd(P.nan_count, (unsigned long long)nans);
        const int total = tile_claim_pair(spike != 0u, b0, b1, s_off, &s_total, &s_base, P.nspk + slot);
        if (spike) {
            const unsigned lt = (1u << lane) - 1u;
            const int pos = s_base + s_off[warp] + __popc(b0 & lt) + __popc(b1 & lt);
            if (spike & 1u) {
                P.spk[pos] = local;
                P.neuron_spikes[local] += 1;
            }
            if (spike & 2u) {
                P.spk[pos + (int)(spike & 1u)] = local + 1;
                P.neuron_spikes[local + 1] += 1;
            }
        }
        if (threadIdx.x == 0 && total) atomicAdd(P.spike_count, (unsigned long long)total);
    }
}

__global__ void k_init_state(const DevPop* pops, const int32_t* tile_pop, float* V, float* m,
                             float* h, float* n, float* g0, float* g1, float* iext, PhiloxKey key) {
    const int tile = blockIdx.x;
    const DevPop& P = pops[tile_pop[tile]];
    const int local = (tile - P.first_tile) * kTile + (int)threadIdx.x;
    const int idx = P.offset + local;
    float v = V[idx], mm = 0.f, hh = 0.f, nn = 0.f;
    if (local < P.n && P.kind == SNN_POP_HH) hh_steady(v, mm, hh, nn);
    if (local < P.n && P.kind == SNN_POP_IZH) {
        hh = izh_r(key, (uint32_t)local, P.tag);          // the neuron's parameter draw r
        mm = fmaf(P.izh[3], hh, P.izh[2]) * v;             // u = b v
    }
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

// Resident CTAs of the step kernel on the current device (cached per device).
static int neuron_grid_cap() {
    static int cap[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (cap[dev] == 0) {
        int sms = 0, per_sm = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_neuron_step, kTile / 2, 0) != cudaSuccess) return 0;
        cap[dev] = std::max(1, sms * per_sm);
    }
    return cap[dev];
}

cudaError_t launch_neuron_step(const NeuronArgs& a, cudaStream_t s) {
    if (a.num_tiles == 0) return cudaSuccess;
    const int cap = neuron_grid_cap();
    if (cap == 0) return cudaErrorUnknown;
    k_neuron_step<<<std::min(a.num_tiles, cap), kTile / 2, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_init_state(const DevPop* pops, int, const int32_t* tile_pop, int num_tiles,
                              float* V, float* m, float* h, float* n, float* g0, float* g1,
                              float* iext, uint64_t seed, cudaStream_t s) {
    if (num_tiles == 0) return cudaSuccess;
    k_init_state<<<num_tiles, kTile, 0, s>>>(pops, tile_pop, V, m, h, n, g0, g1, iext,
                                             PhiloxKey{(uint32_t)seed, (uint32_t)(seed >> 32)});
    return cudaGetLastError();
}

cudaError_t launch_set_epoch_base(unsigned long long* ticket, int num_tiles, cudaStream_t s) {
    k_set_epoch_base<<<1, 1, 0, s>>>(ticket, num_tiles > 0 ? num_tiles : 1);
    return cudaGetLastError();
}

}  // namespace snn
