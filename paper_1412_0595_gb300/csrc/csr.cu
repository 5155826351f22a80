// Compressed-row connectivity on the GPU (Sec. 3 storage): Bernoulli rows
// drawn from the seed (count -> exclusive scan -> fill), validation of caller
// supplied rows, row-length maximum, and the event list of a spike list.
#include "device_math.cuh"
#include "snn_internal.cuh"

namespace snn {

namespace {

constexpr int kThreads = 256;
constexpr int kScanBlock = 1024;     // elements per scan block

// Four Bernoulli bits for posts 4*j4 .. 4*j4+3 of row i (bit e = post 4*j4+e).
__device__ __forceinline__ unsigned edge_bits(PhiloxKey key, uint32_t tag, int64_t i, int64_t j4,
                                              int64_t n_post, unsigned long long thr) {
    const uint4 r = philox_4x32_10(make_uint4((uint32_t)j4, (uint32_t)i, tag, kStreamCsr), key);
    unsigned b = (unsigned)below(r.x, thr) | ((unsigned)below(r.y, thr) << 1) |
                 ((unsigned)below(r.z, thr) << 2) | ((unsigned)below(r.w, thr) << 3);
    const int64_t left = n_post - 4 * j4;      // posts that exist in this group
    if (left < 4) b &= (1u << left) - 1u;
    return b;
}

__global__ void k_csr_count(PhiloxKey key, uint32_t tag, int64_t n_pre, int64_t n_post,
                            unsigned long long thr, int64_t* counts) {
    const int lane = threadIdx.x & 31;
    const int64_t groups = (n_post + 3) / 4;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); i < n_pre; i += warps) {
        int64_t c = 0;
        for (int64_t j4 = lane; j4 < groups; j4 += 32) c += __popc(edge_bits(key, tag, i, j4, n_post, thr));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0) counts[i] = c;
    }
}

__global__ void k_csr_fill(PhiloxKey key, uint32_t tag, int64_t n_pre, int64_t n_post,
                           unsigned long long thr, const int64_t* row_ptr, int32_t* col) {
    const int lane = threadIdx.x & 31;
    const int64_t groups = (n_post + 3) / 4;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); i < n_pre; i += warps) {
        int64_t pos = row_ptr[i];
        for (int64_t base = 0; base < groups; base += 32) {
            const int64_t j4 = base + lane;
            const unsigned b = j4 < groups ? edge_bits(key, tag, i, j4, n_post, thr) : 0u;
            const int cnt = __popc(b);
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            int64_t out = pos + incl - cnt;
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (b & (1u << e)) col[out++] = (int32_t)(4 * j4 + e);
            pos += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
}

// ---- three-phase exclusive scan of int64 (block sums, their scan, apply) ----
__device__ __forceinline__ int64_t block_incl_scan(int64_t v, int64_t* s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x / 32;
        int64_t t = lane < nw ? s_warp[lane] : 0;
        int64_t ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += y;
        }
        if (lane < nw) s_warp[lane] = ti - t;
    }
    __syncthreads();
    const int64_t r = incl + s_warp[warp];
    __syncthreads();
    return r;
}

__global__ void k_scan_sums(const int64_t* in, int64_t n, int64_t* sums) {
    __shared__ int64_t s_warp[32];
    const int64_t base = (int64_t)blockIdx.x * kScanBlock;
    int64_t v = 0;
    for (int e = threadIdx.x; e < kScanBlock; e += blockDim.x)
        if (base + e < n) v += in[base + e];
    const int64_t incl = block_incl_scan(v, s_warp);
    if (threadIdx.x == blockDim.x - 1) sums[blockIdx.x] = incl;
}

__global__ void k_scan_top(int64_t* sums, int64_t nb) {
    __shared__ int64_t s_warp[32];
    __shared__ int64_t s_run;
    if (threadIdx.x == 0) s_run = 0;
    __syncthreads();
    for (int64_t b = 0; b < nb; b += blockDim.x) {
        const int64_t v = b + threadIdx.x < nb ? sums[b + threadIdx.x] : 0;
        const int64_t incl = block_incl_scan(v, s_warp);
        const int64_t run = s_run;
        if (b + threadIdx.x < nb) sums[b + threadIdx.x] = run + incl - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_run = run + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[nb] = s_run;
}

// out[k] = sum_{e < k} in[e] for k in [0, n]; out has n + 1 entries.
__global__ void k_scan_apply(const int64_t* in, int64_t n, const int64_t* sums, int64_t* out) {
    __shared__ int64_t s_warp[32];
    const int64_t base = (int64_t)blockIdx.x * kScanBlock;
    constexpr int kPer = kScanBlock / kThreads;
    int64_t v[kPer];
    int64_t local = 0;
#pragma unroll
    for (int e = 0; e < kPer; ++e) {
        const int64_t k = base + threadIdx.x * kPer + e;
        v[e] = k < n ? in[k] : 0;
        local += v[e];
    }
    const int64_t incl = block_incl_scan(local, s_warp);
    int64_t run = sums[blockIdx.x] + incl - local;
#pragma unroll
    for (int e = 0; e < kPer; ++e) {
        const int64_t k = base + threadIdx.x * kPer + e;
        if (k < n) out[k] = run;
        run += v[e];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = sums[gridDim.x];
}

__global__ void k_validate_csr(const int64_t* row_ptr, const int32_t* col, int32_t n_pre,
                               int32_t n_post, int64_t nnz, uint32_t* error) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); i < n_pre; i += warps) {
        const int64_t b = row_ptr[i], e = row_ptr[i + 1];
        bool bad = (e < b) || b < 0 || e > nnz;
        if (!bad) {
            for (int64_t k = b + lane; k < e; k += 32) {
                const int32_t c = col[k];
                if (c < 0 || c >= n_post || (k > b && col[k - 1] >= c)) bad = true;
            }
        }
        if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(error, kDevErrCsr);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && (row_ptr[0] != 0 || row_ptr[n_pre] != nnz))
        atomicOr(error, kDevErrCsr);
}

__global__ void k_max_row(const int64_t* row_ptr, int32_t n_pre, int32_t* out) {
    int32_t mx = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_pre;
         i += (int64_t)gridDim.x * blockDim.x)
    {
        const int64_t len = row_ptr[i + 1] - row_ptr[i];
        mx = max(mx, len > INT32_MAX ? INT32_MAX : (int32_t)len);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, mx);
}

__global__ void k_row_lengths(const int64_t* row_ptr, const int32_t* spk, int32_t n, int64_t* lens) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) lens[s] = row_ptr[spk[s] + 1] - row_ptr[spk[s]];
}

__global__ void k_event_list(const int64_t* row_ptr, const int32_t* col, const float* w,
                             const int32_t* spk, int32_t n, const int64_t* offsets, int32_t* post_out,
                             float* w_out) {
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x / 32);
    for (int s = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); s < n; s += warps) {
        const int i = spk[s];
        const int64_t b = row_ptr[i], e = row_ptr[i + 1], o = offsets[s];
        for (int64_t k = b + lane; k < e; k += 32) {
            post_out[o + (k - b)] = col[k];
            w_out[o + (k - b)] = w[k];
        }
    }
}

__global__ void k_densify(const int64_t* row_ptr, const int32_t* col, const float* w, int32_t n_pre,
                          int32_t n_post, float* W) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); i < n_pre; i += warps)
        for (int64_t k = row_ptr[i] + lane; k < row_ptr[i + 1]; k += 32) W[i * n_post + col[k]] = w[k];
}

int grid_for(int64_t warps_needed) {
    int64_t b = (warps_needed + (kThreads / 32) - 1) / (kThreads / 32);
    if (b < 1) b = 1;
    if (b > 152 * 16) b = 152 * 16;
    return (int)b;
}

}  // namespace

unsigned long long bernoulli_threshold(double p) {
    if (!(p > 0.0)) return 0ull;
    const double t = nearbyint(p * 4294967296.0);
    if (t >= 4294967296.0) return 4294967296ull;
    return (unsigned long long)t;
}

cudaError_t launch_csr_count(uint64_t seed, uint32_t tag, int64_t n_pre, int64_t n_post,
                             unsigned long long thr, int64_t* counts, cudaStream_t s) {
    if (n_pre == 0) return cudaSuccess;
    const PhiloxKey key{(uint32_t)seed, (uint32_t)(seed >> 32)};
    k_csr_count<<<grid_for(n_pre), kThreads, 0, s>>>(key, tag, n_pre, n_post, thr, counts);
    return cudaGetLastError();
}

cudaError_t launch_csr_fill(uint64_t seed, uint32_t tag, int64_t n_pre, int64_t n_post,
                            unsigned long long thr, const int64_t* row_ptr, int32_t* col, cudaStream_t s) {
    if (n_pre == 0) return cudaSuccess;
    const PhiloxKey key{(uint32_t)seed, (uint32_t)(seed >> 32)};
    k_csr_fill<<<grid_for(n_pre), kThreads, 0, s>>>(key, tag, n_pre, n_post, thr, row_ptr, col);
    return cudaGetLastError();
}

size_t scan_scratch_elems(int64_t n) { return (size_t)((n + kScanBlock - 1) / kScanBlock) + 1; }

cudaError_t launch_scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* scratch, cudaStream_t s) {
    if (n == 0) return cudaMemsetAsync(out, 0, sizeof(int64_t), s);
    const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
    k_scan_sums<<<(unsigned)nb, kThreads, 0, s>>>(in, n, scratch);
    k_scan_top<<<1, 1024, 0, s>>>(scratch, nb);
    k_scan_apply<<<(unsigned)nb, kThreads, 0, s>>>(in, n, scratch, out);
    return cudaGetLastError();
}

cudaError_t launch_validate_csr(const int64_t* row_ptr, const int32_t* col, int32_t n_pre, int32_t n_post,
                                int64_t nnz, uint32_t* error, cudaStream_t s) {
    k_validate_csr<<<grid_for(n_pre), kThreads, 0, s>>>(row_ptr, col, n_pre, n_post, nnz, error);
    return cudaGetLastError();
}

cudaError_t launch_densify(const int64_t* row_ptr, const int32_t* col, const float* w, int32_t n_pre,
                           int32_t n_post, float* W, cudaStream_t s) {
    if (n_pre == 0) return cudaSuccess;
    k_densify<<<grid_for(n_pre), kThreads, 0, s>>>(row_ptr, col, w, n_pre, n_post, W);
    return cudaGetLastError();
}

cudaError_t launch_max_row(const int64_t* row_ptr, int32_t n_pre, int32_t* out, cudaStream_t s) {
    if (n_pre == 0) return cudaSuccess;
    const int blocks = (int)std::min<int64_t>((n_pre + kThreads - 1) / kThreads, 1024);
    k_max_row<<<blocks, kThreads, 0, s>>>(row_ptr, n_pre, out);
    return cudaGetLastError();
}

cudaError_t launch_row_lengths(const int64_t* row_ptr, const int32_t* spk, int32_t n, int64_t* lens,
                               cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_row_lengths<<<(n + kThreads - 1) / kThreads, kThreads, 0, s>>>(row_ptr, spk, n, lens);
    return cudaGetLastError();
}

cudaError_t launch_event_list(const int64_t* row_ptr, const int32_t* col, const float* w, const int32_t* spk,
                              int32_t n, const int64_t* offsets, int32_t* post_out, float* w_out,
                              cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_event_list<<<grid_for(n), kThreads, 0, s>>>(row_ptr, col, w, spk, n, offsets, post_out, w_out);
    return cudaGetLastError();
}

}  // namespace snn
