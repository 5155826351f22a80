// Dense graded projections of the differentiable form (Eq. 2 storage:
// n_pre x n_post weights, row-major).
//
// Forward, every step:   G_q[j] = sum_i w_ij r_i, a matrix-vector product
//   streamed over W.  CTAs take (128 posts, a range of pre rows); each lane
//   sums four posts over its warp's rows, the CTA adds its eight warps in a
//   fixed order and writes a partial row; the last CTA of a post block (a
//   ticket per block) adds the partials in chunk order.  No atomics touch G,
//   so a recomputed step is bit-identical to the first pass.
// Adjoint, per checkpoint segment of L steps:
//   dL/dw_ij += sum_t r_i(t) nu_j(t), nu = dL/dG_q: a rank-L update of the
//   whole matrix, i.e. the product R^T N of the segment's releases (L x n_pre)
//   and dL/dG (n_post x L, time-contiguous).  On the tensor cores (tcgen05):
//   both operands are split into three BF16 parts, x = hi + mid + lo, and the
//   six products hi.hi, hi.mid, mid.hi, hi.lo, lo.hi, mid.mid -- every pair
//   whose weight reaches 2^-24 of the result -- accumulate in FP32 in tensor
//   memory, which keeps an FP32 sum's accuracy.  One CTA per 128 x 128 block of
//   dW: warp 0 streams the K tiles (32 steps) of the six operand tiles into
//   two shared-memory stages with cp.async.bulk, warp 1 issues the MMAs
//   (M = N = 128, K = 16; 12 per K tile), and the eight warps add the
//   accumulator into dW through a shared-memory transposition (row-contiguous
//   global accesses); two CTAs share an SM.  Every wait is bounded; a wait that runs out sets
//   the sticky timeout bit and the CTA drains its copies and MMAs (bounded)
//   and frees its tensor memory before it leaves.  The CUDA-core variant (a
//   shared-memory tiled FP32 product) is kept for comparison.
#include <algorithm>
#include <new>
#include <vector>

#include "snn_internal.cuh"
#include "tc_common.cuh"

namespace snn {

namespace {

using namespace snn::tc;

constexpr int kFwdThreads = 256;
constexpr int kFwdPosts = 128;              // posts per CTA (32 lanes x 4)

// W rows: streamed (evict-first) when the matrix is larger than the L2 share
// it may keep, else through the normal cached path so that it stays resident
// from one step to the next.
template <bool kStream>
__device__ __forceinline__ float4 w_load(const float* p) {
    if constexpr (kStream) return __ldcs(reinterpret_cast<const float4*>(p));
    else return __ldg(reinterpret_cast<const float4*>(p));
}

template <bool kVec, bool kStream>
__global__ void __launch_bounds__(kFwdThreads) k_graded_dense_fwd(const float* __restrict__ W,
                                                                  const float* __restrict__ x, int32_t n_pre,
                                                                  int32_t n_post, int32_t rows_per_chunk,
                                                                  float* __restrict__ Gq, float* __restrict__ part,
                                                                  int64_t ld_part, unsigned* __restrict__ count) {
    __shared__ float4 s_p[kFwdThreads / 32][32];
    __shared__ int s_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int j = (blockIdx.x * 32 + lane) * 4;
    const int i0 = blockIdx.y * rows_per_chunk, i1 = min(n_pre, i0 + rows_per_chunk);
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    if (j < n_post) {
        int i = i0 + warp;
        if constexpr (kVec) {
            // eight rows in flight per lane; the sums stay in ascending row order
            for (; i + 56 < i1; i += 64) {
                float4 w[8];
                float r[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    w[u] = w_load<kStream>(W + (int64_t)(i + 8 * u) * n_post + j);
                    r[u] = __ldg(x + i + 8 * u);
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    acc.x = fmaf(w[u].x, r[u], acc.x);
                    acc.y = fmaf(w[u].y, r[u], acc.y);
                    acc.z = fmaf(w[u].z, r[u], acc.z);
                    acc.w = fmaf(w[u].w, r[u], acc.w);
                }
            }
            for (; i < i1; i += 8) {
                const float4 w = w_load<kStream>(W + (int64_t)i * n_post + j);
                const float r = __ldg(x + i);
                acc.x = fmaf(w.x, r, acc.x);
                acc.y = fmaf(w.y, r, acc.y);
                acc.z = fmaf(w.z, r, acc.z);
                acc.w = fmaf(w.w, r, acc.w);
            }
        } else {
            for (; i < i1; i += 8) {
                const float* row = W + (int64_t)i * n_post + j;
                const float r = __ldg(x + i);
                acc.x = fmaf(row[0], r, acc.x);
                if (j + 1 < n_post) acc.y = fmaf(row[1], r, acc.y);
                if (j + 2 < n_post) acc.z = fmaf(row[2], r, acc.z);
                if (j + 3 < n_post) acc.w = fmaf(row[3], r, acc.w);
            }
        }
    }
    s_p[warp][lane] = acc;
    __syncthreads();
    float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
    if (warp == 0) {
#pragma unroll
        for (int w = 0; w < kFwdThreads / 32; ++w) {
            p.x += s_p[w][lane].x; p.y += s_p[w][lane].y; p.z += s_p[w][lane].z; p.w += s_p[w][lane].w;
        }
    }
    if (gridDim.y == 1) {
        if (warp == 0 && j < n_post) {
            Gq[j] = p.x;
            if (j + 1 < n_post) Gq[j + 1] = p.y;
            if (j + 2 < n_post) Gq[j + 2] = p.z;
            if (j + 3 < n_post) Gq[j + 3] = p.w;
        }
        return;
    }
    if (warp == 0 && j < n_post) *reinterpret_cast<float4*>(part + blockIdx.y * ld_part + j) = p;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(count + blockIdx.x, 1u) == gridDim.y - 1;
    __syncthreads();
    if (!s_last) return;
    // the block's last CTA: every partial row is written and fenced
    __threadfence();
    if (warp == 0 && j < n_post) {
        // eight partial rows in flight, added in chunk order
        float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
        const int nc = (int)gridDim.y;
        for (int c0 = 0; c0 < nc; c0 += 8) {
            float4 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (c0 + u < nc) v[u] = __ldcg(reinterpret_cast<const float4*>(part + (int64_t)(c0 + u) * ld_part + j));
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (c0 + u < nc) {
                    g.x += v[u].x; g.y += v[u].y; g.z += v[u].z; g.w += v[u].w;
                }
        }
        Gq[j] = g.x;
        if (j + 1 < n_post) Gq[j + 1] = g.y;
        if (j + 2 < n_post) Gq[j + 2] = g.z;
        if (j + 3 < n_post) Gq[j + 3] = g.w;
    }
    if (threadIdx.x == 0) count[blockIdx.x] = 0u;       // ready for the next step
}

// ---- weight gradient on the tensor cores --------------------------------------
constexpr int kGK = 32;                       // K elements (steps) per tile
constexpr int kGTile = kRows * kGK;           // 4096 BF16 = 8 KiB
constexpr int kGStages = 2;                   // 2 x 48 KiB: two CTAs per SM overlap loads, MMAs and epilogues
constexpr int kGStageBytes = 6 * kGTile * 2;  // three A parts + three B parts
constexpr uint32_t kGSbo = (kGK / 8) * 128;
constexpr int kGThreads = 256;
constexpr uint32_t kGIdesc = idesc_bf16(kRows, kRows);
// (A part, B part) pairs of the six products, largest first
__constant__ int c_pair_a[6] = {0, 0, 1, 0, 2, 1};
__constant__ int c_pair_b[6] = {0, 1, 0, 2, 0, 1};

// Eight consecutive K elements of one row are one 16-byte row of a core
// matrix in the tiled layout: each thread splits eight values and writes each
// part with one 16-byte store.
__device__ __forceinline__ void split8_store(const float (&x)[8], uint16_t* dst, int64_t part_elems) {
    uint16_t hi[8], mid[8], lo[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) split3(x[u], hi[u], mid[u], lo[u]);
    auto pack = [](const uint16_t (&h)[8]) {
        return make_uint4((uint32_t)h[0] | ((uint32_t)h[1] << 16), (uint32_t)h[2] | ((uint32_t)h[3] << 16),
                          (uint32_t)h[4] | ((uint32_t)h[5] << 16), (uint32_t)h[6] | ((uint32_t)h[7] << 16));
    };
    *reinterpret_cast<uint4*>(dst) = pack(hi);
    *reinterpret_cast<uint4*>(dst + part_elems) = pack(mid);
    *reinterpret_cast<uint4*>(dst + 2 * part_elems) = pack(lo);
}

// A[i][t] = R[t][i] (for the network: a step's releases of the pre
// population), 3 parts, tiled (mp x kp).  Grid (mp / 256, kp / 8): a thread
// takes eight steps of one pre index; pre index fastest across the warp
// (coalesced reads of each step's row).
__global__ void __launch_bounds__(256) k_grad_split_a(const float* __restrict__ R, int64_t ldr, int32_t m, int32_t L,
                                                      int64_t mp, int64_t kp, uint16_t* __restrict__ A) {
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x, t0 = (int64_t)blockIdx.y * 8;
    if (i >= mp) return;
    float x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) x[u] = (i < m && t0 + u < L) ? R[(t0 + u) * ldr + i] : 0.0f;
    split8_store(x, A + tiled_offset(i, t0, kp / kGK, kGK), mp * kp);
}

// B[j][t] = N[j][t] (for the network: dL/dG of a post over the segment,
// time-contiguous), 3 parts, tiled (np x kp).  A thread takes eight steps of
// one post, steps fastest across the warp (coalesced reads of a row of N).
__global__ void __launch_bounds__(256) k_grad_split_b(const float* __restrict__ N, int64_t ldn, int32_t n, int32_t L,
                                                      int64_t np, int64_t kp, uint16_t* __restrict__ B) {
    const int64_t per_row = kp / 8;
    const int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (e >= np * per_row) return;
    const int64_t j = e / per_row, t0 = (e % per_row) * 8;
    float x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) x[u] = (j < n && t0 + u < L) ? N[j * ldn + t0 + u] : 0.0f;
    split8_store(x, B + tiled_offset(j, t0, kp / kGK, kGK), np * kp);
}

__global__ void __launch_bounds__(kGThreads, 1)
    k_dense_grad_mma(const uint16_t* __restrict__ A, const uint16_t* __restrict__ B, int64_t mp, int64_t np,
                     int64_t kp, int32_t m, int32_t n, float* D, int64_t ldd, uint32_t* error, uint32_t spin_limit) {
    extern __shared__ __align__(1024) unsigned char s_raw[];
    __shared__ __align__(8) unsigned long long s_full[kGStages], s_done[kGStages];
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    const int nt = blockIdx.x, mt = blockIdx.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_k = (int)(kp / kGK);
    const int64_t a_part = mp * kp, b_part = np * kp;

    if (warp == 0) {
        // one accumulator of 128 FP32 columns x 128 lanes
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(smem_u32(&s_tmem))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < kGStages; ++i) {
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

    // stage layout: A parts 0..2, then B parts 0..2
    auto stage_ptr = [&](int st, int slot) { return s_raw + (size_t)st * kGStageBytes + (size_t)slot * kGTile * 2; };
    if (threadIdx.x == 0) {
        for (int i = 0; i < n_k; ++i) {
            const int st = i % kGStages;
            if (i >= kGStages && !mbar_wait(smem_u32(&s_done[st]), (i / kGStages - 1) & 1, spin_limit)) {
                atomicOr(error, kDevErrTimeout);
                s_fail = 1;
                break;
            }
            const uint32_t bar = smem_u32(&s_full[st]);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                         "r"((uint32_t)kGStageBytes) : "memory");
            for (int p = 0; p < 3; ++p) {
                bulk_copy(stage_ptr(st, p), A + p * a_part + ((int64_t)mt * n_k + i) * kGTile, kGTile * 2, bar);
                bulk_copy(stage_ptr(st, 3 + p), B + p * b_part + ((int64_t)nt * n_k + i) * kGTile, kGTile * 2, bar);
            }
        }
    } else if (threadIdx.x == 32) {
        bool ok = true;
        for (int i = 0; i < n_k; ++i) {
            const int st = i % kGStages;
            if (!mbar_wait(smem_u32(&s_full[st]), (i / kGStages) & 1, spin_limit)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int ks = 0; ks < kGK / 16; ++ks)
                for (int pp = 0; pp < 6; ++pp) {
                    const uint64_t da = smem_desc(smem_u32(stage_ptr(st, c_pair_a[pp])) + ks * 256, 128, kGSbo);
                    const uint64_t db = smem_desc(smem_u32(stage_ptr(st, 3 + c_pair_b[pp])) + ks * 256, 128, kGSbo);
                    mma_bf16(tmem, da, db, kGIdesc, (i | ks | pp) != 0);
                }
            mma_commit(smem_u32(&s_done[st]));
        }
        if (ok && !mbar_wait(smem_u32(&s_done[(n_k - 1) % kGStages]), ((n_k - 1) / kGStages) & 1, spin_limit))
            ok = false;
        if (!ok) {
            atomicOr(error, kDevErrTimeout);
            s_fail = 1;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (s_fail && threadIdx.x == 0) {
        for (int st = 0; st < kGStages; ++st)
            for (uint32_t par = 0; par < 2; ++par) {
                mbar_wait(smem_u32(&s_full[st]), par, spin_limit);
                mbar_wait(smem_u32(&s_done[st]), par, spin_limit);
            }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    __syncwarp();
    if (!s_fail) {
        // every copy has landed and every MMA is done: the stages hold the
        // transposition tile (128 x kTileLd floats)
        float* st = reinterpret_cast<float*>(s_raw);
        tmem_tile_to_smem(tmem, st, warp, lane);
        __syncthreads();
        const int64_t i0 = (int64_t)mt * kRows, j0 = (int64_t)nt * kRows;
        const int rows = (int)(m - i0 < kRows ? m - i0 : kRows), cols = (int)(n - j0 < kRows ? n - j0 : kRows);
        const bool vec = (ldd & 3) == 0 && (reinterpret_cast<uintptr_t>(D) & 15) == 0;
        smem_tile_to_global<false>(st, D + i0 * ldd + j0, ldd, rows, cols, nullptr, vec, warp, lane);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem) : "memory");
    }
}

// CUDA-core variant: 64 x 64 blocks of dW, 4 x 4 per thread, the segment's
// steps in chunks of 16 staged in shared memory.
constexpr int kRB = 64, kRT = 16;

__global__ void __launch_bounds__(256) k_dense_grad_rows(const float* __restrict__ R, int64_t ldr, int32_t m,
                                                         const float* __restrict__ N, int64_t ldn, int32_t n,
                                                         int32_t L, float* D, int64_t ldd) {
    __shared__ __align__(16) float s_r[kRT][kRB];
    __shared__ __align__(16) float s_n[kRT][kRB + 4];    // rows of 272 bytes keep float4 reads aligned
    const int i0 = blockIdx.y * kRB, j0 = blockIdx.x * kRB;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc[4][4] = {};
    for (int t0 = 0; t0 < L; t0 += kRT) {
        for (int e = threadIdx.x; e < kRT * kRB; e += 256) {
            const int tt = e / kRB, ii = e % kRB;           // releases: pre index fastest
            const int t = t0 + tt, i = i0 + ii;
            s_r[tt][ii] = (t < L && i < m) ? R[(int64_t)t * ldr + i] : 0.0f;
            const int jj = e / kRT, tn = e % kRT;           // N: step fastest
            const int j = j0 + jj, t2 = t0 + tn;
            s_n[tn][jj] = (t2 < L && j < n) ? N[(int64_t)j * ldn + t2] : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int tt = 0; tt < kRT; ++tt) {
            const float4 a = *reinterpret_cast<const float4*>(&s_r[tt][ty * 4]);
            const float4 b = *reinterpret_cast<const float4*>(&s_n[tt][tx * 4]);
            const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int i = i0 + ty * 4 + u;
        if (i >= m) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int j = j0 + tx * 4 + v;
            if (j < n) D[(int64_t)i * ldd + j] += acc[u][v];
        }
    }
}

}  // namespace

int dense_fwd_chunks(int32_t n_pre, int32_t n_post, int sm_count) {
    const int blocks = (n_post + kFwdPosts - 1) / kFwdPosts;
    int chunks = (4 * sm_count + blocks - 1) / blocks;          // about four CTAs per SM
    chunks = std::min(chunks, std::max(1, n_pre / 64));          // at least eight rows per warp
    chunks = std::min(chunks, 64);                               // a short reduction for narrow matrices
    return std::max(1, chunks);
}

cudaError_t launch_graded_dense_fwd(const float* W, const float* x, int32_t n_pre, int32_t n_post, float* Gq,
                                    float* part, int64_t ld_part, unsigned* count, int32_t chunks, bool stream,
                                    cudaStream_t s) {
    if (n_post == 0) return cudaSuccess;
    const int rows = (n_pre + chunks - 1) / chunks;
    const dim3 grid((unsigned)((n_post + kFwdPosts - 1) / kFwdPosts), (unsigned)chunks);
    if ((n_post & 3) == 0) {
        if (stream)
            k_graded_dense_fwd<true, true><<<grid, kFwdThreads, 0, s>>>(W, x, n_pre, n_post, rows, Gq, part, ld_part,
                                                                        count);
        else
            k_graded_dense_fwd<true, false><<<grid, kFwdThreads, 0, s>>>(W, x, n_pre, n_post, rows, Gq, part, ld_part,
                                                                         count);
    } else {
        k_graded_dense_fwd<false, false><<<grid, kFwdThreads, 0, s>>>(W, x, n_pre, n_post, rows, Gq, part, ld_part,
                                                                      count);
    }
    return cudaGetLastError();
}

void dense_grad_sizes(int32_t n_pre, int32_t n_post, int32_t K, int64_t* mp, int64_t* np, int64_t* kp) {
    *mp = (int64_t)(n_pre + kRows - 1) / kRows * kRows;
    *np = (int64_t)(n_post + kRows - 1) / kRows * kRows;
    *kp = (int64_t)(K + kGK - 1) / kGK * kGK;
}

cudaError_t launch_dense_grad(const DenseGradArgs& g, cudaStream_t s) {
    if (g.m == 0 || g.n == 0 || g.L == 0) return cudaSuccess;
    if (g.engine == 0) {
        const dim3 grid((unsigned)((g.n + kRB - 1) / kRB), (unsigned)((g.m + kRB - 1) / kRB));
        k_dense_grad_rows<<<grid, 256, 0, s>>>(g.R, g.ldr, g.m, g.N, g.ldn, g.n, g.L, g.D, g.ldd);
        return cudaGetLastError();
    }
    int64_t mp, np, kp;
    dense_grad_sizes(g.m, g.n, g.L, &mp, &np, &kp);
    k_grad_split_a<<<dim3((unsigned)(mp / 256 + (mp % 256 != 0)), (unsigned)(kp / 8)), 256, 0, s>>>(g.R, g.ldr, g.m,
                                                                                                g.L, mp, kp, g.A);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t nb = np * (kp / 8);
    k_grad_split_b<<<(unsigned)((nb + 255) / 256), 256, 0, s>>>(g.N, g.ldn, g.n, g.L, np, kp, g.B);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t smem = (size_t)kGStages * kGStageBytes;
    e = cudaFuncSetAttribute(k_dense_grad_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)(np / kRows), (unsigned)(mp / kRows));
    k_dense_grad_mma<<<grid, kGThreads, smem, s>>>(g.A, g.B, mp, np, kp, g.m, g.n, g.D, g.ldd, g.error, g.spin_limit);
    return cudaGetLastError();
}

}  // namespace snn

struct snn_dense_grad {
    snn::Alloc mem;
    std::vector<void*> owned;
    uint16_t *A = nullptr, *B = nullptr;
    size_t a_cap = 0, b_cap = 0;
    uint32_t* error = nullptr;
    uint32_t spin_limit = 1u << 22;
};

namespace {

snn_status dg_cuda(cudaError_t e, const char* what) { return e == cudaSuccess ? SNN_OK : snn::cuda_fail(e, what); }

// Grows one of the handle's part buffers to `need` BF16 elements.
snn_status dg_grow(snn_dense_grad* h, uint16_t** p, size_t* cap, size_t need, cudaStream_t s) {
    if (need <= *cap) return SNN_OK;
    if (*p) {
        snn_status st = dg_cuda(cudaStreamSynchronize(s), "synchronize");
        if (st != SNN_OK) return st;
        h->owned.erase(std::find(h->owned.begin(), h->owned.end(), (void*)*p));
        h->mem.put(*p);
        *p = nullptr;
        *cap = 0;
    }
    void* q = h->mem.get(need * sizeof(uint16_t));
    if (!q) return snn::fail(SNN_ERR_OOM, "device allocation failed: gradient operand parts");
    h->owned.push_back(q);
    *p = static_cast<uint16_t*>(q);
    *cap = need;
    return SNN_OK;
}

}  // namespace

extern "C" {

snn_status snn_dense_grad_create(const snn_allocator* alloc, void* stream, snn_dense_grad** out) {
    if (!out) return snn::fail(SNN_ERR_INVALID_ARG, "dense gradient: out is NULL");
    auto* h = new (std::nothrow) snn_dense_grad();
    if (!h) return snn::fail(SNN_ERR_OOM, "host allocation failed");
    if (alloc) {
        h->mem.a = *alloc;
        h->mem.have = true;
    }
    h->mem.stream = stream;
    h->error = static_cast<uint32_t*>(h->mem.get(sizeof(uint32_t)));
    snn_status st = h->error ? SNN_OK : snn::fail(SNN_ERR_OOM, "device allocation failed: error word");
    if (st == SNN_OK) {
        h->owned.push_back(h->error);
        st = dg_cuda(cudaMemsetAsync(h->error, 0, sizeof(uint32_t), (cudaStream_t)stream), "clear");
    }
    if (st == SNN_OK) st = dg_cuda(cudaStreamSynchronize((cudaStream_t)stream), "synchronize");
    if (st != SNN_OK) {
        snn_dense_grad_destroy(h);
        return st;
    }
    *out = h;
    return SNN_OK;
}

snn_status snn_dense_grad_destroy(snn_dense_grad* h) {
    if (!h) return SNN_OK;
    cudaDeviceSynchronize();
    for (void* p : h->owned) h->mem.put(p);
    delete h;
    return SNN_OK;
}

snn_status snn_dense_grad_run(snn_dense_grad* h, const float* R, int64_t ldr, const float* N, int64_t ldn,
                              int32_t m, int32_t n, int32_t K, float* D, int64_t ldd, int32_t engine, void* stream) {
    if (!h || m < 0 || n < 0 || K < 0 || K > snn::kMaxSeg || (engine != 0 && engine != 1))
        return snn::fail(SNN_ERR_INVALID_ARG, "dense gradient: bad sizes or engine");
    if (m == 0 || n == 0 || K == 0) return SNN_OK;
    if (!R || !N || !D || ldr < m || ldn < K || ldd < n)
        return snn::fail(SNN_ERR_INVALID_ARG, "dense gradient: bad pointers or strides");
    cudaStream_t s = (cudaStream_t)stream;
    snn::DenseGradArgs g{};
    g.R = R; g.ldr = ldr; g.N = N; g.ldn = ldn; g.m = m; g.n = n; g.L = K; g.D = D; g.ldd = ldd;
    g.engine = engine;
    g.error = h->error;
    g.spin_limit = h->spin_limit;
    if (engine == 1) {
        int64_t mp, np, kp;
        snn::dense_grad_sizes(m, n, K, &mp, &np, &kp);
        snn_status st = dg_grow(h, &h->A, &h->a_cap, (size_t)(3 * mp * kp), s);
        if (st == SNN_OK) st = dg_grow(h, &h->B, &h->b_cap, (size_t)(3 * np * kp), s);
        if (st != SNN_OK) return st;
    }
    g.A = h->A;
    g.B = h->B;
    return dg_cuda(snn::launch_dense_grad(g, s), "dense gradient");
}

snn_status snn_dense_grad_check(snn_dense_grad* h, void* stream) {
    if (!h) return snn::fail(SNN_ERR_INVALID_ARG, "dense gradient is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t err = 0;
    snn_status st = dg_cuda(cudaMemcpyAsync(&err, h->error, sizeof(err), cudaMemcpyDeviceToHost, s), "read error word");
    if (st == SNN_OK) st = dg_cuda(cudaStreamSynchronize(s), "synchronize");
    if (st != SNN_OK) return st;
    if (err & snn::kDevErrTimeout) return snn::fail(SNN_ERR_TIMEOUT, "dense gradient: a bounded wait ran out");
    return SNN_OK;
}

}  // extern "C"
