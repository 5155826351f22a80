// Allocation-free variant of the connectivity row builder.
//
// snn_csr_bernoulli_rows takes scratch memory for its scan from an allocator.
// Some callers cannot allocate device memory at the moment they need
// connectivity: code whose device memory is all owned by a pool or a budget
// it must not step outside, and loops that must not call cudaMalloc /
// cudaFree at all (cudaFree, for one, may wait for the whole device).  This
// entry point serves them: the per-row counts go straight into the caller's
// row_ptr, and the only scratch (the per-block sums of the scan) lives in a
// fixed file-scope device array.  It calls no cudaMalloc, cudaFree or
// allocating routine; it waits on its own stream only, to hand the total
// back on the host.
#include <mutex>

#include "snn_internal.cuh"

namespace snn {

namespace {

constexpr int kRowsPerBlock = 1024;     // rows per scan block
constexpr int kScanThreads = 256;       // 4 rows per thread
constexpr int64_t kMaxScanBlocks = (int64_t)SNN_NOALLOC_MAX_ROWS / kRowsPerBlock;
constexpr int kMaxDevices = 64;

// Block sums of the scan (+ the total).  One copy per GPU that loads the
// library, kept until the process exits; shared by every call on that GPU.
static __device__ __align__(256) long long g_noalloc_block_sums[kMaxScanBlocks + 1];

std::mutex g_mu;
struct ScratchSlot {
    void* ctx;            // the device's context the address belongs to
    long long* ptr;
};
ScratchSlot g_scratch[kMaxDevices] = {};

typedef int (*CtxGetCurrentFn)(void**);

// The calling thread's current context (the device's primary context for
// runtime-API callers; null while the runtime has not bound one to this
// thread yet), through the driver entry point the runtime exposes, so the
// library needs no link to the driver library.
snn_status current_context(void** ctx) {
    static CtxGetCurrentFn fn = nullptr;
    *ctx = nullptr;
    if (!fn) {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !f)
            return fail(SNN_ERR_CUDA, "cuCtxGetCurrent entry point not found");
        fn = reinterpret_cast<CtxGetCurrentFn>(f);
    }
    if (fn(ctx) != 0) return fail(SNN_ERR_CUDA, "cuCtxGetCurrent failed");
    return SNN_OK;
}

// Device address of the scratch array on the current device.  The set-up
// runs once per device, with that device current: the first call looks the
// address up (this may load the library's module onto the device).  The
// address is kept with the device's context, so after cudaDeviceReset (or any
// reset of the primary context, which may move module variables) the next
// call looks it up again.
snn_status scratch_address(long long** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "get device");
    if (dev < 0 || dev >= kMaxDevices) return fail(SNN_ERR_INVALID_ARG, "device index out of range");
    void* ctx = nullptr;
    snn_status st = current_context(&ctx);
    if (st != SNN_OK) return st;
    std::lock_guard<std::mutex> lock(g_mu);
    ScratchSlot& slot = g_scratch[dev];
    if (!ctx || !slot.ptr || slot.ctx != ctx) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_block_sums);   // binds the primary context if none was current
        if (e != cudaSuccess) return cuda_fail(e, "scratch address");
        st = current_context(&ctx);
        if (st != SNN_OK) return st;
        if (!ctx) return fail(SNN_ERR_CUDA, "no current context after the scratch lookup");
        slot.ptr = static_cast<long long*>(p);
        slot.ctx = ctx;
    }
    *out = slot.ptr;
    return SNN_OK;
}

__device__ __forceinline__ long long block_scan_incl(long long v, long long* s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x / 32;
        const long long t = lane < nw ? s_warp[lane] : 0;
        long long u = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, u, o);
            if (lane >= o) u += y;
        }
        if (lane < nw) s_warp[lane] = u - t;
    }
    __syncthreads();
    const long long r = x + s_warp[warp];
    __syncthreads();
    return r;
}

// sums[b] = sum of counts in block b (counts live at row_ptr[1 .. n]).
__global__ void k_na_block_sums(const int64_t* counts, int64_t n, long long* sums) {
    __shared__ long long s_warp[32];
    const int64_t base = (int64_t)blockIdx.x * kRowsPerBlock;
    long long v = 0;
    for (int e = threadIdx.x; e < kRowsPerBlock; e += blockDim.x)
        if (base + e < n) v += counts[base + e];
    const long long incl = block_scan_incl(v, s_warp);
    if (threadIdx.x == blockDim.x - 1) sums[blockIdx.x] = incl;
}

// Exclusive scan of the nb block sums in place; sums[nb] = total.
__global__ void k_na_scan_sums(long long* sums, int64_t nb) {
    __shared__ long long s_warp[32];
    __shared__ long long s_run;
    if (threadIdx.x == 0) s_run = 0;
    __syncthreads();
    for (int64_t b = 0; b < nb; b += blockDim.x) {
        const long long v = b + threadIdx.x < nb ? sums[b + threadIdx.x] : 0;
        const long long incl = block_scan_incl(v, s_warp);
        const long long run = s_run;
        if (b + threadIdx.x < nb) sums[b + threadIdx.x] = run + incl - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_run = run + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[nb] = s_run;
}

// In place: row_ptr[1 + k] <- sum_{e <= k} count_e, row_ptr[0] <- 0.
__global__ void k_na_rows_inclusive(int64_t* row_ptr, int64_t n, const long long* sums) {
    __shared__ long long s_warp[32];
    constexpr int kPer = kRowsPerBlock / kScanThreads;
    int64_t* counts = row_ptr + 1;
    const int64_t base = (int64_t)blockIdx.x * kRowsPerBlock + (int64_t)threadIdx.x * kPer;
    long long v[kPer];
    long long local = 0;
#pragma unroll
    for (int e = 0; e < kPer; ++e) {
        v[e] = base + e < n ? counts[base + e] : 0;
        local += v[e];
    }
    const long long incl = block_scan_incl(local, s_warp);
    long long run = sums[blockIdx.x] + incl - local;
#pragma unroll
    for (int e = 0; e < kPer; ++e) {
        run += v[e];
        if (base + e < n) counts[base + e] = run;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) row_ptr[0] = 0;
}

}  // namespace

}  // namespace snn

using namespace snn;

extern "C" snn_status snn_csr_bernoulli_rows_noalloc(uint64_t seed, uint32_t tag, int64_t n_pre, int64_t n_post,
                                                     double p, int64_t* row_ptr, int64_t* nnz, void* stream) {
    if (n_pre < 0 || n_post < 0 || n_post >= (int64_t(1) << 31) || !(p >= 0.0) || p > 1.0 || !row_ptr || !nnz)
        return fail(SNN_ERR_INVALID_ARG, "bad sizes, probability or pointers");
    if (n_pre > (int64_t)SNN_NOALLOC_MAX_ROWS)
        return fail(SNN_ERR_SIZE, "n_pre exceeds SNN_NOALLOC_MAX_ROWS (16777216) rows of the fixed scratch array");
    long long* sums = nullptr;
    snn_status st = scratch_address(&sums);
    if (st != SNN_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (n_pre == 0) {
        e = cudaMemsetAsync(row_ptr, 0, sizeof(int64_t), s);
    } else {
        const int64_t nb = (n_pre + kRowsPerBlock - 1) / kRowsPerBlock;
        // counts of row i land in row_ptr[1 + i]; every scratch entry read
        // below (sums[0 .. nb]) is written first by this call.
        e = launch_csr_count(seed, tag, n_pre, n_post, bernoulli_threshold(p), row_ptr + 1, s);
        if (e == cudaSuccess) {
            k_na_block_sums<<<(unsigned)nb, kScanThreads, 0, s>>>(row_ptr + 1, n_pre, sums);
            k_na_scan_sums<<<1, 1024, 0, s>>>(sums, nb);
            k_na_rows_inclusive<<<(unsigned)nb, kScanThreads, 0, s>>>(row_ptr, n_pre, sums);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(nnz, row_ptr + n_pre, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "draw rows without allocation");
    return SNN_OK;
}
