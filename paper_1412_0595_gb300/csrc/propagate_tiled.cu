// Post-tiled propagation for compressed rows with long rows and many posts.
//
// One global float atomic per synapse caps the row-per-warp kernel well below
// HBM bandwidth when rows are long (100 rows x 500,000 synapses per step).
// Here a CTA owns one tile of P consecutive post neurons and a group of
// spiking rows: it streams, for each row, only the segment whose post indices
// fall in its tile (segment bounds come from a split table computed once at
// creation: split[i][T] = first synapse of row i with post >= T * P), adds
// s * w into a shared-memory accumulator, and flushes the tile to the
// conductance with one 16-byte vector reduction per four posts.  Post indices
// are distinct within a row, so the CTA walks the rows one at a time with a
// barrier between rows and adds with plain read-modify-writes (no shared
// atomics, and a fixed summation order within the tile).  Global atomics drop
// from one per synapse to P / 4 per (tile, row group).
#include "snn_internal.cuh"

namespace snn {

namespace {

constexpr int kThreads = 256;
constexpr int kUnroll = 4;

__global__ void k_row_splits(const int64_t* row_ptr, const int32_t* col, int32_t n_pre, int32_t n_tiles,
                             int32_t P, int64_t* split) {
    const int64_t total = (int64_t)n_pre * (n_tiles + 1);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / (n_tiles + 1);
        const int64_t T = e - i * (n_tiles + 1);
        const int64_t key = T * (int64_t)P;
        int64_t lo = row_ptr[i], hi = row_ptr[i + 1];      // first k in [lo, hi) with col[k] >= key
        while (lo < hi) {
            const int64_t mid = lo + ((hi - lo) >> 1);
            if (col[mid] < key) lo = mid + 1;
            else hi = mid;
        }
        split[e] = lo;
    }
}

__global__ void __launch_bounds__(kThreads) k_propagate_tiled(const DevProj* qp, const unsigned long long* ticket,
                                                               int32_t num_tiles) {
    extern __shared__ float s_acc[];
    const DevProj& q = *qp;
    const int slot = (int)((*ticket / (unsigned long long)num_tiles + 1ull) & 1ull);
    const int ns = q.nspk[slot];
    if (ns == 0) return;
    const int nt = q.n_ptiles, P = q.ptile;
    // rows per item so that there are about four items per CTA
    const int64_t want = 4ll * gridDim.x;
    const int64_t g_rows = ((int64_t)ns * nt + want - 1) / want;
    const int G = g_rows < 1 ? 1 : (int)g_rows;
    const int groups = (ns + G - 1) / G;
    const int64_t items = (int64_t)groups * nt;
    const float s = q.scale;
    for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
        const int T = (int)(item % nt);
        const int grp = (int)(item / nt);
        const int post0 = T * P;
        const int width = min(P, q.n_post - post0);
        for (int j = threadIdx.x; j < width; j += kThreads) s_acc[j] = 0.0f;
        __syncthreads();
        const int r_end = min(ns, (grp + 1) * G);
        for (int r = grp * G; r < r_end; ++r) {
            const int64_t* sp = q.split + (int64_t)q.spk[r] * (nt + 1) + T;
            const int64_t beg = sp[0], end = sp[1];
            const int64_t k0 = beg & ~int64_t(3);
            for (int64_t kb = k0 + 4 * threadIdx.x; kb < end; kb += 4 * kThreads * kUnroll) {
                int4 c4[kUnroll];
                float4 w4[kUnroll];
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) {
                    const int64_t k = kb + (int64_t)u * 4 * kThreads;
                    if (k < end) {
                        c4[u] = __ldcs(reinterpret_cast<const int4*>(q.col + k));
                        w4[u] = __ldcs(reinterpret_cast<const float4*>(q.w + k));
                    }
                }
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) {
                    const int64_t k = kb + (int64_t)u * 4 * kThreads;
                    if (k < end) {
                        if (k >= beg) s_acc[c4[u].x - post0] += s * w4[u].x;
                        if (k + 1 >= beg && k + 1 < end) s_acc[c4[u].y - post0] += s * w4[u].y;
                        if (k + 2 >= beg && k + 2 < end) s_acc[c4[u].z - post0] += s * w4[u].z;
                        if (k + 3 >= beg && k + 3 < end) s_acc[c4[u].w - post0] += s * w4[u].w;
                    }
                }
            }
            __syncthreads();                     // the next row may hit the same posts
        }
        float* g = q.g + post0;
        if ((width & 3) == 0) {
            for (int j = 4 * threadIdx.x; j < width; j += 4 * kThreads) {
                const float4 v = *reinterpret_cast<const float4*>(s_acc + j);
                if (v.x != 0.f || v.y != 0.f || v.z != 0.f || v.w != 0.f)
                    atomicAdd(reinterpret_cast<float4*>(g + j), v);
            }
        } else {
            for (int j = threadIdx.x; j < width; j += kThreads)
                if (s_acc[j] != 0.f) atomicAdd(g + j, s_acc[j]);
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_row_splits(const int64_t* row_ptr, const int32_t* col, int32_t n_pre, int32_t n_tiles, int32_t P,
                              int64_t* split, cudaStream_t s) {
    const int64_t total = (int64_t)n_pre * (n_tiles + 1);
    if (total == 0) return cudaSuccess;
    const int blocks = (int)std::min<int64_t>((total + kThreads - 1) / kThreads, 4096);
    k_row_splits<<<blocks, kThreads, 0, s>>>(row_ptr, col, n_pre, n_tiles, P, split);
    return cudaGetLastError();
}

cudaError_t launch_propagate_tiled(const DevProj* q, int32_t P, const unsigned long long* ticket, int32_t num_tiles,
                                   int blocks, cudaStream_t s) {
    const size_t smem = sizeof(float) * (size_t)P;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_propagate_tiled, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_propagate_tiled<<<blocks, kThreads, smem, s>>>(q, ticket, std::max(1, num_tiles));
    return cudaGetLastError();
}

}  // namespace snn
