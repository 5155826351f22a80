// Dense spike delivery for many network instances that share one dense
// projection (Sec. 3, Eq. 2 storage), on the tensor cores.
//
// For B instances, G[b][j] += s_b * sum_i S[b][i] W[i][j] with S the 0/1
// spike matrix of the step: one matrix product per step instead of one row
// read per spike and instance.  S is exact in BF16.  W is split once into
// three BF16 parts, W = hi + mid + lo (each part the BF16 rounding of what
// the previous parts left), which carry W's 24 significant bits, and the
// three products accumulate in FP32 in tensor memory: the result has the
// accuracy of an FP32 sum.
//
// Layout: operands are stored K-major in the tensor core's canonical
// no-swizzle form, tile by tile (128 rows x 64 K-elements = 16 KiB, core
// matrices of 8 rows x 16 bytes, 8 of them along K per 8-row group), so each
// tile is one contiguous bulk copy into shared memory.
//
// Kernel (one CTA of 256 threads per 256 x 128 output tile and K range):
// one thread (warp 0) streams the K tiles of two 128-row S tiles and of the
// three W parts into three shared-memory stages with cp.async.bulk
// (completion on an mbarrier); another (warp 1) issues, as each stage lands,
// its tcgen05.mma chain (M = 128, N = 128, K = 16 per instruction; 18 per K
// tile: 3 K steps x 3 parts x 2 row tiles, the W tiles shared by both) into
// two 128-column FP32 accumulators in tensor memory; tcgen05.commit
// releases a stage when its MMAs are done.  The eight
// warps then read each accumulator with tcgen05.ld into shared memory and add
// s_b times its rows to G, lanes along a row (contiguous global accesses).  When
// the output has few tiles the K range is split over CTAs (split-K), which
// then add with atomics.  Every wait is bounded: a wait that runs out sets
// the sticky timeout bit, and the CTA still waits (bounded) for its copies
// and MMAs and frees its tensor memory before it leaves.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "snn_internal.cuh"
#include "tc_common.cuh"

namespace {

constexpr int kTM = 128;              // output rows (instances) per tile
constexpr int kTN = 128;              // output columns (posts) per tile
constexpr int kTK = 48;               // K elements (pre neurons) per tile
constexpr int kTileElems = kTM * kTK; // 6144 BF16 = 12 KiB (same for the W tiles: kTN = kTM)
constexpr int kStages = 3;            // shared-memory stages of the operand pipeline (3 x 60 KiB)
constexpr uint32_t kSbo = (kTK / 8) * 128;   // bytes between 8-row groups of core matrices
constexpr int kStageBytes = 5 * kTileElems * 2;   // two S tiles + three W-part tiles
constexpr int kThreadsMma = 256;

static_assert(kTN == kTM, "S and W tiles share one tile shape");

using namespace snn::tc;

// Device-side choice between the two delivery paths inside a time step (so
// one captured sequence serves every spike count): gate 0 always runs, gate 1
// runs when the step's spikes (spk_off[B]) reach thr, gate 2 when they do not.
__device__ __forceinline__ bool gated_off(int32_t gate, const int32_t* spk_off, int32_t B, int64_t thr) {
    if (gate == 0) return false;
    const bool dense = (int64_t)spk_off[B] >= thr;
    return gate == 1 ? !dense : dense;
}

// Element offset of (row, k) inside the tiled K-major layout with `kt` K tiles per row band.
__host__ __device__ __forceinline__ int64_t tiled_offset(int64_t row, int64_t k, int64_t kt) {
    return snn::tc::tiled_offset(row, k, kt, kTK);
}

// W (n_pre x n_post, row-major FP32) -> three BF16 parts of W^T (post-major),
// tiled; zero padding up to (np, kp).
__global__ void k_split_weights(const float* W, int32_t n_pre, int32_t n_post, int64_t np, int64_t kp,
                                uint16_t* parts) {
    const int64_t total = np * kp, kt = kp / kTK;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t n = e / kp, k = e % kp;
        const float w = (n < n_post && k < n_pre) ? W[k * n_post + n] : 0.0f;
        uint16_t hi, mid, lo;
        split3(w, hi, mid, lo);
        const int64_t o = tiled_offset(n, k, kt);
        parts[o] = hi;
        parts[total + o] = mid;
        parts[2 * total + o] = lo;
    }
}

// Row b of S (bp x kp, tiled), one CTA per row: zero (16-byte stores of 8
// consecutive K elements, which are contiguous in the tiled layout), then
// 1.0 at every spike of instance b (rows b >= B stay zero).
__global__ void k_build_spikes(const int32_t* spk_off, const int32_t* spk, int32_t B, int32_t n_pre, int64_t kp,
                               uint16_t* S, uint32_t* error, int32_t gate, int64_t thr) {
    if (gated_off(gate, spk_off, B, thr)) return;
    const int b = blockIdx.x;
    const int64_t kt = kp / kTK;
    for (int64_t k8 = threadIdx.x; k8 < kp / 8; k8 += blockDim.x)
        *reinterpret_cast<uint4*>(S + tiled_offset(b, 8 * k8, kt)) = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    if (b >= B) return;
    const int32_t beg = spk_off[b], end = spk_off[b + 1];
    for (int32_t s = beg + threadIdx.x; s < end; s += blockDim.x) {
        const int32_t i = spk[s];
        if (i < 0 || i >= n_pre) {
            atomicOr(error, snn::kDevErrCsr);     // an index outside the pre population
            continue;
        }
        S[tiled_offset(b, i, kt)] = 0x3F80;   // BF16 1.0
    }
}

constexpr uint32_t kIdesc = idesc_bf16(kTM, kTN);

__global__ void __launch_bounds__(kThreadsMma, 1)
    k_dense_batch_mma(const uint16_t* __restrict__ S, const uint16_t* __restrict__ parts, int64_t np, int64_t kp,
                      int32_t B, int32_t n_post, const float* __restrict__ scale, float* G, int64_t ldg,
                      uint32_t* error, uint32_t spin_limit, int32_t k_per_cta, const int32_t* spk_off,
                      int32_t gate, int64_t thr) {
    if (gated_off(gate, spk_off, B, thr)) return;          // uniform over the CTA, before any barrier
    extern __shared__ __align__(1024) unsigned char s_raw[];
    __shared__ __align__(8) unsigned long long s_full[kStages], s_done[kStages];
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    const int nt = blockIdx.x, mt2 = blockIdx.y;      // row tiles 2 mt2 and 2 mt2 + 1
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t kt = kp / kTK;
    const int k0 = blockIdx.z * k_per_cta;
    const int k1 = min((int)kt, k0 + k_per_cta);
    const bool split = gridDim.z > 1;
    const int64_t part_elems = np * kp;

    if (warp == 0) {
        // two accumulators of 128 FP32 columns x 128 lanes
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(&s_tmem))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < kStages; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_full[i])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_done[i])) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;

    auto stage_ptr = [&](int st, int part) { return s_raw + (size_t)st * kStageBytes + (size_t)part * kTileElems * 2; };
    const int n_k = k1 - k0;
    if (threadIdx.x == 0) {
        // producer: tile i goes into stage i % kStages once the MMAs of tile
        // i - kStages (the stage's previous use) have completed
        for (int i = 0; i < n_k; ++i) {
            const int st = i % kStages;
            if (i >= kStages && !mbar_wait(smem_u32(&s_done[st]), (i / kStages - 1) & 1, spin_limit)) {
                atomicOr(error, snn::kDevErrTimeout);
                s_fail = 1;
                break;
            }
            const int kc = k0 + i;
            const uint32_t bar = smem_u32(&s_full[st]);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"((uint32_t)kStageBytes)
                         : "memory");
            for (int h = 0; h < 2; ++h)
                bulk_copy(stage_ptr(st, h), S + ((int64_t)(2 * mt2 + h) * kt + kc) * kTileElems, kTileElems * 2, bar);
            for (int p = 0; p < 3; ++p)
                bulk_copy(stage_ptr(st, 2 + p), parts + p * part_elems + ((int64_t)nt * kt + kc) * kTileElems,
                          kTileElems * 2, bar);
        }
    } else if (threadIdx.x == 32) {
        // MMA issuer: as soon as a stage has landed, its 3 x 2 x kTK / 16 MMAs
        bool ok = true;
        for (int i = 0; i < n_k; ++i) {
            const int st = i % kStages;
            if (!mbar_wait(smem_u32(&s_full[st]), (i / kStages) & 1, spin_limit)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int ks = 0; ks < kTK / 16; ++ks)          // K = 16 per MMA: two core matrices
                for (int p = 0; p < 3; ++p) {
                    const uint64_t db = smem_desc(smem_u32(stage_ptr(st, 2 + p)) + ks * 256, 128, kSbo);
                    for (int h = 0; h < 2; ++h) {
                        const uint64_t da = smem_desc(smem_u32(stage_ptr(st, h)) + ks * 256, 128, kSbo);
                        mma_bf16(tmem + (uint32_t)(h * kTN), da, db, kIdesc, (i | ks | p) != 0);
                    }
                }
            mma_commit(smem_u32(&s_done[st]));
        }
        // the accumulators are complete when the range's last tile's MMAs are
        if (ok && !mbar_wait(smem_u32(&s_done[(n_k - 1) % kStages]), ((n_k - 1) / kStages) & 1, spin_limit))
            ok = false;
        if (!ok) {
            atomicOr(error, snn::kDevErrTimeout);
            s_fail = 1;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (s_fail && threadIdx.x == 0) {
        // wait (bounded) for whatever may still be in flight into this CTA
        for (int st = 0; st < kStages; ++st)
            for (uint32_t par = 0; par < 2; ++par) {
                mbar_wait(smem_u32(&s_full[st]), par, spin_limit);
                mbar_wait(smem_u32(&s_done[st]), par, spin_limit);
            }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    __syncwarp();                                         // tcgen05.ld is warp-collective
    if (!s_fail) {
        // every copy has landed and every MMA is done: the stages hold the
        // transposition tile; accumulator h covers instances 128 (2 mt2 + h) ..
        float* st = reinterpret_cast<float*>(s_raw);
        const int64_t j0 = (int64_t)nt * kTN;
        const int cols = (int)(n_post - j0 < kTN ? n_post - j0 : kTN);
        const bool vec = (ldg & 3) == 0 && (reinterpret_cast<uintptr_t>(G) & 15) == 0;
        for (int h = 0; h < 2; ++h) {
            const int64_t b0 = (int64_t)(2 * mt2 + h) * kTM;
            const int64_t left = (int64_t)B - b0;
            const int rows = (int)(left <= 0 ? 0 : (left < kTM ? left : kTM));
            tmem_tile_to_smem(tmem + (uint32_t)(h * kTN), st, warp, lane);
            __syncthreads();
            if (rows > 0) {
                if (split) smem_tile_to_global<true>(st, G + b0 * ldg + j0, ldg, rows, cols, scale + b0, vec, warp, lane);
                else smem_tile_to_global<false>(st, G + b0 * ldg + j0, ldg, rows, cols, scale + b0, vec, warp, lane);
            }
            __syncthreads();                              // the tile is read before the next one is written
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
    }
}

// CUDA-core delivery (the plain path for comparison): one CTA per (instance,
// 1024 posts); each thread sums its four posts over the instance's spikes.
__global__ void __launch_bounds__(256) k_dense_batch_rows(const float* __restrict__ W, int32_t n_post,
                                                          const int32_t* spk_off, const int32_t* spk,
                                                          const float* scale, float* G, int64_t ldg, int32_t B,
                                                          int32_t gate, int64_t thr) {
    if (gated_off(gate, spk_off, B, thr)) return;
    const int b = blockIdx.y;
    const int j = (blockIdx.x * 256 + threadIdx.x) * 4;
    if (j >= n_post) return;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    const bool vec = (n_post & 3) == 0;
    for (int32_t s = spk_off[b]; s < spk_off[b + 1]; ++s) {
        const float* row = W + (int64_t)spk[s] * n_post + j;
        if (vec) {
            const float4 w = __ldg(reinterpret_cast<const float4*>(row));
            a0 += w.x; a1 += w.y; a2 += w.z; a3 += w.w;
        } else {
            a0 += row[0];
            if (j + 1 < n_post) a1 += row[1];
            if (j + 2 < n_post) a2 += row[2];
            if (j + 3 < n_post) a3 += row[3];
        }
    }
    float* g = G + (int64_t)b * ldg + j;
    const float sb = scale[b];
    g[0] += sb * a0;
    if (j + 1 < n_post) g[1] += sb * a1;
    if (j + 2 < n_post) g[2] += sb * a2;
    if (j + 3 < n_post) g[3] += sb * a3;
}

}  // namespace

struct snn_dense_batch {
    snn::Alloc mem;
    std::vector<void*> owned;      // device allocations, freed by snn_dense_batch_destroy
    int32_t n_pre = 0, n_post = 0;
    int64_t np = 0, kp = 0;
    uint16_t* parts = nullptr;     // 3 x np x kp BF16, tiled
    float* W = nullptr;            // n_pre x n_post FP32 (CUDA-core path)
    uint16_t* S = nullptr;         // spike matrix, bp_cap x kp BF16, tiled
    int64_t bp_cap = 0;
    uint32_t* error = nullptr;
    uint32_t spin_limit = 1u << 22;
    int sm_count = 0;
    bool smem_set = false;
};

using snn::fail;

namespace {

template <typename T>
snn_status dalloc(snn_dense_batch* h, T** p, size_t n, const char* what) {
    *p = static_cast<T*>(h->mem.get(sizeof(T) * std::max<size_t>(n, 1)));
    if (!*p) return fail(SNN_ERR_OOM, std::string("device allocation failed: ") + what);
    h->owned.push_back(*p);
    return SNN_OK;
}

void release(snn_dense_batch* h) {
    cudaDeviceSynchronize();
    for (void* p : h->owned) h->mem.put(p);
    h->owned.clear();
}

snn_status cuda(cudaError_t e, const char* what) {
    return e == cudaSuccess ? SNN_OK : snn::cuda_fail(e, what);
}

snn_status check_error(snn_dense_batch* h, cudaStream_t s) {
    uint32_t err = 0;
    snn_status st = cuda(cudaMemcpyAsync(&err, h->error, sizeof(err), cudaMemcpyDeviceToHost, s), "read error word");
    if (st == SNN_OK) st = cuda(cudaStreamSynchronize(s), "synchronize");
    if (st != SNN_OK) return st;
    if (err & snn::kDevErrTimeout) return fail(SNN_ERR_TIMEOUT, "tensor-core delivery: a bounded wait ran out");
    if (err & snn::kDevErrCsr) return fail(SNN_ERR_INVALID_ARG, "spike index outside the pre population");
    return SNN_OK;
}

}  // namespace

extern "C" {

snn_status snn_dense_batch_create(const float* W, int32_t n_pre, int32_t n_post, int32_t w_on_device,
                                  const snn_allocator* alloc, void* stream, snn_dense_batch** out) {
    if (!out || !W || n_pre < 1 || n_post < 1 || (int64_t)n_pre * n_post > (int64_t(1) << 31))
        return fail(SNN_ERR_INVALID_ARG, "dense batch: bad weights or sizes");
    cudaStream_t s = (cudaStream_t)stream;
    auto* h = new (std::nothrow) snn_dense_batch();
    if (!h) return fail(SNN_ERR_OOM, "host allocation failed");
    if (alloc) {
        h->mem.a = *alloc;
        h->mem.have = true;
    }
    h->mem.stream = stream;
    h->n_pre = n_pre;
    h->n_post = n_post;
    h->np = (n_post + kTN - 1) / kTN * kTN;
    h->kp = (n_pre + kTK - 1) / kTK * kTK;
    int dev = 0;
    snn_status st = cuda(cudaGetDevice(&dev), "get device");
    if (st == SNN_OK) st = cuda(cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, dev), "SMs");
    if (st == SNN_OK) st = dalloc(h, &h->parts, (size_t)(3 * h->np * h->kp), "weight parts");
    if (st == SNN_OK) st = dalloc(h, &h->W, (size_t)n_pre * n_post + 4, "weights");
    if (st == SNN_OK) st = dalloc(h, &h->error, 1, "error word");
    if (st == SNN_OK)
        st = cuda(cudaMemcpyAsync(h->W, W, sizeof(float) * (size_t)n_pre * n_post,
                                  w_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s), "copy weights");
    if (st == SNN_OK) st = cuda(cudaMemsetAsync(h->error, 0, sizeof(uint32_t), s), "clear");
    if (st == SNN_OK) {
        const int64_t total = h->np * h->kp;
        k_split_weights<<<(int)std::min<int64_t>((total + 255) / 256, 8192), 256, 0, s>>>(h->W, n_pre, n_post, h->np,
                                                                                         h->kp, h->parts);
        st = cuda(cudaGetLastError(), "split weights");
    }
    if (st == SNN_OK) st = cuda(cudaStreamSynchronize(s), "synchronize");
    if (st != SNN_OK) {
        release(h);
        delete h;
        return st;
    }
    *out = h;
    return SNN_OK;
}

snn_status snn_dense_batch_destroy(snn_dense_batch* h) {
    if (!h) return SNN_OK;
    release(h);
    delete h;
    return SNN_OK;
}

snn_status snn_dense_batch_deliver(snn_dense_batch* h, int32_t B, const int32_t* spk_off, const int32_t* spk,
                                   const float* scale, float* G, int64_t ldg, int32_t engine, void* stream) {
    if (!h || B < 0 || !spk_off || !scale || !G || ldg < h->n_post || (engine != 0 && engine != 1))
        return fail(SNN_ERR_INVALID_ARG, "dense batch: bad arguments");
    if (B == 0) return SNN_OK;
    cudaStream_t s = (cudaStream_t)stream;
    snn_status st = SNN_OK;
    if (engine == 1 && (st = snn::dense_batch_reserve(h, B, s)) != SNN_OK) return st;
    return cuda(snn::dense_batch_launch(h, B, spk_off, spk, scale, G, ldg, engine, 0, s), "dense delivery");
}

snn_status snn_dense_batch_check(snn_dense_batch* h, void* stream) {
    if (!h) return fail(SNN_ERR_INVALID_ARG, "dense batch is NULL");
    return check_error(h, (cudaStream_t)stream);
}

}  // extern "C"

namespace snn {

// Spike-matrix capacity for B instances (allocates; not inside a capture).
snn_status dense_batch_reserve(snn_dense_batch* h, int32_t B, cudaStream_t s) {
    const int64_t bp = (int64_t)(B + 2 * kTM - 1) / (2 * kTM) * (2 * kTM);   // whole pairs of row tiles
    snn_status st = SNN_OK;
    if (bp > h->bp_cap) {
        if (h->S) {
            if ((st = cuda(cudaStreamSynchronize(s), "synchronize")) != SNN_OK) return st;
            h->owned.erase(std::find(h->owned.begin(), h->owned.end(), (void*)h->S));
            h->mem.put(h->S);
        }
        h->S = nullptr;
        if ((st = dalloc(h, &h->S, (size_t)(bp * h->kp), "spike matrix")) != SNN_OK) return st;
        h->bp_cap = bp;
    }
    if (!h->smem_set) {
        const size_t smem = kStages * (size_t)kStageBytes;
        if ((st = cuda(cudaFuncSetAttribute(k_dense_batch_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                       "shared memory")) != SNN_OK)
            return st;
        h->smem_set = true;
    }
    return SNN_OK;
}

// G[b] += scale[b] * (S W)[b] for the spike lists (spk_off, spk) of B
// instances: engine 0 CUDA cores, 1 tensor cores, 2 both launched with the
// device-side gate (tensor cores when the spikes reach `thr`).  The tensor
// path needs dense_batch_reserve(h, >= B) first; nothing here allocates or
// synchronises, so it may be captured.
cudaError_t dense_batch_launch(snn_dense_batch* h, int32_t B, const int32_t* spk_off, const int32_t* spk,
                               const float* scale, float* G, int64_t ldg, int32_t engine, int64_t thr, cudaStream_t s) {
    if (B == 0) return cudaSuccess;
    if (engine == 0 || engine == 2) {
        const dim3 grid((unsigned)((h->n_post + 1023) / 1024), (unsigned)B);
        k_dense_batch_rows<<<grid, 256, 0, s>>>(h->W, h->n_post, spk_off, spk, scale, G, ldg, B, engine == 2 ? 2 : 0,
                                                thr);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess || engine == 0) return e;
    }
    const int64_t bp = (int64_t)(B + 2 * kTM - 1) / (2 * kTM) * (2 * kTM);   // whole pairs of row tiles
    if (bp > h->bp_cap || !h->smem_set) return cudaErrorInvalidValue;
    const int32_t gate = engine == 2 ? 1 : 0;
    k_build_spikes<<<(unsigned)bp, 128, 0, s>>>(spk_off, spk, B, h->n_pre, h->kp, h->S, h->error, gate, thr);
    const size_t smem = kStages * (size_t)kStageBytes;
    // split the K range only when the output has fewer than half as many
    // tiles as SMs (measured: a split that only evens out the waves costs
    // more in its atomic epilogue than the idle SMs of the last wave)
    const int64_t tiles = (h->np / kTN) * (bp / (2 * kTM)), kt = h->kp / kTK;
    int64_t ksplit = tiles * 2 > h->sm_count ? 1 : std::min<int64_t>(kt, (h->sm_count + tiles - 1) / tiles);
    const int k_per = (int)((kt + ksplit - 1) / ksplit);
    ksplit = (kt + k_per - 1) / k_per;
    const dim3 grid((unsigned)(h->np / kTN), (unsigned)(bp / (2 * kTM)), (unsigned)ksplit);
    k_dense_batch_mma<<<grid, kThreadsMma, smem, s>>>(h->S, h->parts, h->np, h->kp, B, h->n_post, scale, G, ldg,
                                                      h->error, h->spin_limit, k_per, spk_off, gate, thr);
    return cudaGetLastError();
}

}  // namespace snn
