// Spike compaction shared by the step kernels.  A warp ballot and a CTA scan
// order a tile's spikes by neuron index; the tile then claims a contiguous
// slot range of its population's list with one atomic add.  Tiles never wait
// for each other, so the list is ascending within each tile and the tiles'
// ranges follow completion order (the C-ABI sorts when it hands the list out).
// List lengths are double-buffered by step parity: step e counts into slot
// e & 1 and clears slot (e + 1) & 1, which the previous step's consumers have
// finished reading by then.
#pragma once

#include "snn_internal.cuh"

namespace snn {

// Called by every thread of the CTA (kTile threads) with its spike flag.
// Returns the tile's spike total; s_off[warp] receives warp offsets within
// the tile and *s_base the claimed start in the population list.
// A tile without spikes costs one barrier.
__device__ __forceinline__ int tile_claim(bool spike, unsigned ballot, int* s_off, int* s_total, int* s_base,
                                          int32_t* nspk_slot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (__syncthreads_count(spike) == 0) return 0;
    if (lane == 0) s_off[warp] = __popc(ballot);
    __syncthreads();
    if (warp == 0) {
        const int c = lane < kTile / 32 ? s_off[lane] : 0;
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane < kTile / 32) s_off[lane] = incl - c;
        if (lane == 31) {
            *s_total = incl;
            *s_base = incl ? atomicAdd(nspk_slot, incl) : 0;
        }
    }
    __syncthreads();
    return *s_total;
}

// The same for a CTA of kTile / 2 threads that each hold two neurons of the
// tile (neurons 2 t and 2 t + 1): b0 / b1 are the warp's ballots of the
// pairs' first / second halves, so a warp covers 64 neurons in the order
// (lane, half).  Returns the tile's spike total; s_off[warp] receives warp
// offsets within the tile and *s_base the claimed start in the list.
__device__ __forceinline__ int tile_claim_pair(bool any, unsigned b0, unsigned b1, int* s_off, int* s_total,
                                               int* s_base, int32_t* nspk_slot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int kWarps = kTile / 64;
    if (__syncthreads_count(any) == 0) return 0;
    if (lane == 0) s_off[warp] = __popc(b0) + __popc(b1);
    __syncthreads();
    if (warp == 0) {
        const int c = lane < kWarps ? s_off[lane] : 0;
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane < kWarps) s_off[lane] = incl - c;
        if (lane == 31) {
            *s_total = incl;
            *s_base = incl ? atomicAdd(nspk_slot, incl) : 0;
        }
    }
    __syncthreads();
    return *s_total;
}

}  // namespace snn
