// Spike propagation over compressed-row and dense connectivity (Sec. 3).
//
// One launch per time step covers every projection.  The work is a flat list
// of warp items built on the device from the spike counts the neuron kernel
// left behind (no host round trip):
//   compressed rows: one item = (spiking row, chunk of `chunk` synapses); the
//     warp streams col/w with 16-byte cache-streaming loads from HBM and adds
//     s * w into the post conductance with fire-and-forget reductions (the
//     post array stays resident in L2);
//   dense rows: one item = (32 spiking rows, 128 consecutive posts); each lane
//     sums four posts over the 32 rows in registers and issues one 16-byte
//     vector reduction.
// CTAs stride over the item list (grid sized to the SM count), so the same
// captured launch serves any spike count, including none.
#include "snn_internal.cuh"

namespace snn {

namespace {

constexpr int kPropThreads = 256;
constexpr int kDenseRows = 32;     // spiking rows per dense item
constexpr int kDensePosts = 128;   // posts per dense item (32 lanes x 4)

__device__ __forceinline__ int64_t items_of(const DevProj& q, int slot) {
    if (q.mode != 0) return 0;                    // post-tiled rows have their own kernels
    const int64_t ns = q.nspk[slot];
    if (q.layout == SNN_LAYOUT_CSR) return ns * q.chunks;
    return ((ns + kDenseRows - 1) / kDenseRows) * q.chunks;
}

__device__ __forceinline__ void csr_item(const DevProj& q, int64_t r, int chunk, int lane) {
    const int64_t si = r / q.chunks;
    const int64_t c = r - si * q.chunks;
    const int i = q.spk[si];
    const int64_t row_beg = q.row_ptr[i], row_end = q.row_ptr[i + 1];
    const int64_t beg = row_beg + c * chunk;
    if (beg >= row_end) return;
    const int64_t end = min(row_end, beg + chunk);
    const float s = q.scale;
    float* __restrict__ g = q.g;
    // col / w are padded to a multiple of 4 entries, so aligned 16-byte loads
    // that start at or before `end` stay inside the allocation.
    for (int64_t k = (beg & ~int64_t(3)) + 4 * lane; k < end; k += 128) {
        const int4 c4 = __ldcs(reinterpret_cast<const int4*>(q.col + k));
        const float4 w4 = __ldcs(reinterpret_cast<const float4*>(q.w + k));
        if (k >= beg) atomicAdd(g + c4.x, s * w4.x);
        if (k + 1 >= beg && k + 1 < end) atomicAdd(g + c4.y, s * w4.y);
        if (k + 2 >= beg && k + 2 < end) atomicAdd(g + c4.z, s * w4.z);
        if (k + 3 >= beg && k + 3 < end) atomicAdd(g + c4.w, s * w4.w);
    }
}

__device__ __forceinline__ void dense_item(const DevProj& q, int64_t r, int lane, int slot) {
    const int64_t sb = r / q.chunks;
    const int pb = (int)(r - sb * q.chunks);
    const int ns = q.nspk[slot];
    const int s_beg = (int)sb * kDenseRows;
    const int cnt = min(ns, s_beg + kDenseRows) - s_beg;          // spiking rows of this item (<= 32)
    const int n_post = q.n_post;
    const int j = pb * kDensePosts + 4 * lane;
    const bool in = j < n_post;
    // lane t holds the t-th spiking row, so the weight loads below do not wait
    // on a spike-list load; eight rows are in flight per lane
    const int my_row = lane < cnt ? q.spk[s_beg + lane] : 0;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    const float sc = q.scale;
    if ((n_post & 3) == 0) {
#pragma unroll 8
        for (int t = 0; t < cnt; ++t) {
            const int row = __shfl_sync(0xffffffffu, my_row, t);
            if (in) {
                const float4 w4 = __ldcs(reinterpret_cast<const float4*>(q.w + (int64_t)row * n_post + j));
                a0 += w4.x; a1 += w4.y; a2 += w4.z; a3 += w4.w;
            }
        }
        if (in) atomicAdd(reinterpret_cast<float4*>(q.g + j), make_float4(sc * a0, sc * a1, sc * a2, sc * a3));
    } else {
#pragma unroll 4
        for (int t = 0; t < cnt; ++t) {
            const int row = __shfl_sync(0xffffffffu, my_row, t);
            if (in) {
                const float* w = q.w + (int64_t)row * n_post + j;
                a0 += w[0];
                if (j + 1 < n_post) a1 += w[1];
                if (j + 2 < n_post) a2 += w[2];
                if (j + 3 < n_post) a3 += w[3];
            }
        }
        if (in) {
            atomicAdd(q.g + j, sc * a0);
            if (j + 1 < n_post) atomicAdd(q.g + j + 1, sc * a1);
            if (j + 2 < n_post) atomicAdd(q.g + j + 2, sc * a2);
            if (j + 3 < n_post) atomicAdd(q.g + j + 3, sc * a3);
        }
    }
}

}  // namespace

__global__ void __launch_bounds__(kPropThreads) k_propagate(const PropArgs a) {
    extern __shared__ int64_t s_pref[];   // n_projs + 1 item offsets
    const int np = a.n_projs;
    // list-length slot of the step whose spikes are delivered
    const int slot = (int)((*a.ticket / (unsigned long long)a.num_tiles + 1ull) & 1ull);
    // Item offsets of every projection (warp 0 scans 32 projections at a time).
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        int64_t run = 0;
        for (int b = 0; b < np; b += 32) {
            const int q = b + lane;
            const int64_t v = q < np ? items_of(a.projs[q], slot) : 0;
            int64_t incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (q < np) s_pref[q] = run + incl - v;
            run += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (lane == 0) s_pref[np] = run;
    }
    __syncthreads();
    const int64_t total = s_pref[np];
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (kPropThreads / 32);
    int q = 0;
    for (int64_t item = (int64_t)blockIdx.x * (kPropThreads / 32) + (threadIdx.x >> 5); item < total;
         item += warps) {
        while (s_pref[q + 1] <= item) ++q;      // items ascend, so q only moves forward
        const DevProj& Q = a.projs[q];
        const int64_t r = item - s_pref[q];
        if (Q.layout == SNN_LAYOUT_CSR) csr_item(Q, r, a.chunk, lane);
        else dense_item(Q, r, lane, slot);
    }
}

cudaError_t propagate_occupancy(int* per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_propagate, kPropThreads, 0);
}

cudaError_t launch_propagate(const PropArgs& a, int blocks, cudaStream_t s) {
    if (a.n_projs == 0 || a.num_tiles == 0) return cudaSuccess;
    const size_t smem = sizeof(int64_t) * (size_t)(a.n_projs + 1);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_propagate, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_propagate<<<blocks, kPropThreads, smem, s>>>(a);
    return cudaGetLastError();
}

// Synaptic events since reset: sum over pre neurons of spikes x row length.
__global__ void k_count_events(const DevProj* projs, unsigned long long* out) {
    const DevProj& q = projs[blockIdx.y];
    unsigned long long acc = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < q.n_pre; i += gridDim.x * blockDim.x) {
        const long long c = q.pre_count[i];
        if (c) acc += (unsigned long long)(c * (q.layout == SNN_LAYOUT_CSR ? q.row_ptr[i + 1] - q.row_ptr[i]
                                                                          : (int64_t)q.n_post));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, acc);
}

cudaError_t launch_count_events(const DevProj* projs, int n_projs, unsigned long long* out, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess || n_projs == 0) return e;
    k_count_events<<<dim3(64, n_projs), 256, 0, s>>>(projs, out);
    return cudaGetLastError();
}

int dense_rows_per_item() { return kDenseRows; }
int dense_posts_per_item() { return kDensePosts; }

}  // namespace snn
