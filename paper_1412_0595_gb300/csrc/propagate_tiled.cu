// Post-tiled propagation for compressed rows with long rows and many posts.
//
// One global float atomic per synapse caps the row-per-warp kernel well below
// HBM bandwidth when rows are long (100 rows x 500,000 synapses per step).
// Here a CTA owns one tile of P consecutive post neurons and a group of
// spiking rows: it streams, for each row, only the segment whose post indices
// fall in its tile (segment bounds come from a split table computed once at
// creation: split[i][T] = first synapse of row i with post >= T * P), adds
// s * w into a shared-memory accumulator, and flushes the tile to the
// conductance with one 16-byte vector reduction per four posts.
//
// The segments move global -> shared by the bulk-copy engine (cp.async.bulk,
// completion counted on an mbarrier).  One piece is the segment of one row in
// one tile, widened to 16-byte boundaries; one thread keeps kStages - 1
// pieces in flight while the CTA adds the current one with plain shared-memory
// read-modify-writes (the posts of a row are distinct) and a barrier between
// pieces keeps the rows in order (a fixed summation order within the tile).
// Several CTAs share an SM, so one CTA's adds and barriers overlap another's
// copies.  Every mbarrier wait is bounded; a wait that runs out sets the
// sticky timeout bit, and the CTA waits (bounded) for its own copies in flight
// before it leaves.
#include "snn_internal.cuh"

namespace snn {

namespace {

constexpr int kThreads = 256;

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

constexpr int kStages = 3;
constexpr int kChunk = kPostTile + 8;     // synapses per piece: a whole segment of a row in one tile (+ alignment)
constexpr int kMaxPieces = 256;           // pieces described per batch
constexpr int kMaxRowsPerItem = 64;
struct Piece {
    int64_t lo;                           // first synapse copied (16-byte aligned)
    int32_t n;                            // synapses copied (multiple of 4, at most kChunk)
    int32_t b_off, e_off;                 // the valid synapses are [lo + b_off, lo + e_off)
    int32_t post0;                        // first post of the tile
    int32_t last;                         // 1 on the last piece of a tile (row group x tile)
    int32_t pad;
};
static_assert(sizeof(Piece) == 32, "Piece is 32 bytes");

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    return done != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint32_t limit) {
    for (uint32_t it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Issues the copies of one piece into stage buffers (one thread).
__device__ __forceinline__ void issue_piece(const Piece& pc, const int32_t* col, const float* w, int32_t* s_col,
                                            float* s_w, uint32_t bar) {
    const uint32_t bytes = (uint32_t)pc.n * 4u;
    // the stage was last read through the generic proxy; order that before the async-proxy writes
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(2u * bytes) : "memory");
    if (bytes) {
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     ::"r"(smem_u32(s_col)), "l"(col + pc.lo), "r"(bytes), "r"(bar) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     ::"r"(smem_u32(s_w)), "l"(w + pc.lo), "r"(bytes), "r"(bar) : "memory");
    }
}

__global__ void __launch_bounds__(kThreads) k_propagate_tiled(const DevProj* qp, const unsigned long long* ticket,
                                                                  int32_t num_tiles, uint32_t* error,
                                                                  uint32_t spin_limit) {
    extern __shared__ __align__(128) unsigned char s_raw[];
    const DevProj& q = *qp;
    const int slot = (int)((*ticket / (unsigned long long)num_tiles + 1ull) & 1ull);
    const int ns = q.nspk[slot];
    if (ns == 0) return;
    const int nt = q.n_ptiles, P = q.ptile;
    // layout: stage indices [kStages][kChunk] | stage weights [kStages][kChunk] |
    // pieces [kMaxPieces] | accumulator [P] | full [kStages]
    int32_t* s_col = reinterpret_cast<int32_t*>(s_raw);
    float* s_w = reinterpret_cast<float*>(s_col + kStages * kChunk);
    Piece* s_piece = reinterpret_cast<Piece*>(s_w + kStages * kChunk);
    float* s_acc = reinterpret_cast<float*>(s_piece + kMaxPieces);
    unsigned long long* s_full = reinterpret_cast<unsigned long long*>(s_acc + P);
    __shared__ int s_n_pieces, s_next_item, s_abort_flag;
    volatile int& s_abort = s_abort_flag;  // written by any thread, read after barriers

    // rows per item so that there are about four items per CTA
    const int64_t want = 4ll * gridDim.x;
    const int64_t g_rows = ((int64_t)ns * nt + want - 1) / want;
    const int G = g_rows < 1 ? 1 : (g_rows > kMaxRowsPerItem ? kMaxRowsPerItem : (int)g_rows);
    const int groups = (ns + G - 1) / G;
    const int64_t items = (int64_t)groups * nt;
    const float sc = q.scale;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    if (threadIdx.x == 0) {
        for (int st = 0; st < kStages; ++st)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(s_full + st)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    for (int j = threadIdx.x; j < P; j += kThreads) s_acc[j] = 0.0f;
    __syncthreads();

    uint32_t used = 0;                    // pieces of earlier batches (global piece g uses stage g % kStages)
    int64_t item = blockIdx.x;            // next item to describe
    while (item < items) {
        // ---- describe a batch of pieces (warp 0), whole items only ----------
        if (warp == 0) {
            int n = 0;
            int64_t it = item;
            for (; it < items; it += gridDim.x) {
                const int T = (int)(it % nt), grp = (int)(it / nt);
                const int r0 = grp * G, r1 = min(ns, r0 + G);
                if (n + (r1 - r0) + 1 > kMaxPieces) break;           // at most one piece per row
                const int n_item0 = n;
                for (int rb = r0; rb < r1; rb += 32) {
                    const int r = rb + lane;
                    int64_t beg = 0, end = 0;
                    if (r < r1) {
                        const int64_t* sp = q.split + (int64_t)q.spk[r] * (nt + 1) + T;
                        beg = sp[0];
                        end = sp[1];
                    }
                    const int np = end > beg ? 1 : 0;
                    const unsigned mask = __ballot_sync(0xffffffffu, np);
                    if (np) {
                        Piece pc;
                        pc.lo = beg & ~int64_t(3);
                        pc.n = (int)(((end + 3) & ~int64_t(3)) - pc.lo);
                        pc.b_off = (int)(beg - pc.lo);
                        pc.e_off = (int)(end - pc.lo);
                        pc.post0 = T * P;
                        pc.last = 0;
                        pc.pad = 0;
                        s_piece[n + __popc(mask & ((1u << lane) - 1u))] = pc;
                    }
                    n += __popc(mask);
                }
                if (n == n_item0) {               // a tile without synapses still ends (an empty flush)
                    if (lane == 0) {
                        Piece pc{0, 0, 0, 0, T * P, 0, 0};
                        s_piece[n] = pc;
                    }
                    ++n;
                }
                __syncwarp();                     // the item's pieces are written
                if (lane == 0) s_piece[n - 1].last = 1;
                __syncwarp();
            }
            if (lane == 0) {
                s_n_pieces = n;
                s_next_item = (int)((it - item) / gridDim.x);
            }
        }
        __syncthreads();
        const int n = s_n_pieces;
        item += (int64_t)s_next_item * gridDim.x;
        // ---- stream the pieces -----------------------------------------------
        if (threadIdx.x == 0)
            for (int i = 0; i < kStages - 1 && i < n; ++i) {
                const uint32_t st = (used + i) % kStages;
                issue_piece(s_piece[i], q.col, q.w, s_col + st * kChunk, s_w + st * kChunk, smem_u32(s_full + st));
            }
        int i_abort = -1;
        for (int i = 0; i < n; ++i) {
            // piece i + kStages - 1 goes into the stage piece i - 1 used (freed by the last barrier)
            if (threadIdx.x == 0 && i + kStages - 1 < n) {
                const uint32_t st = (used + i + kStages - 1) % kStages;
                issue_piece(s_piece[i + kStages - 1], q.col, q.w, s_col + st * kChunk, s_w + st * kChunk,
                            smem_u32(s_full + st));
            }
            const uint32_t g = used + (uint32_t)i, st = g % kStages;
            const bool ok = mbar_wait_bounded(smem_u32(s_full + st), (g / kStages) & 1u, spin_limit);
            if (!ok) {
                atomicOr(error, kDevErrTimeout);
                s_abort = 1;
            }
            const Piece pc = s_piece[i];
            if (ok) {
                // consecutive threads take consecutive synapses; a thread's posts
                // are distinct (one row), so it gathers before it stores
                const int32_t* c_st = s_col + st * kChunk;
                const float* w_st = s_w + st * kChunk;
                float* acc = s_acc - pc.post0;
                for (int e = threadIdx.x; e < pc.n; e += 4 * kThreads) {
                    int ci[4];
                    float av[4], wv[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int x = e + u * kThreads;
                        const bool v = x >= pc.b_off && x < pc.e_off;
                        ci[u] = v ? c_st[x] : -1;
                        wv[u] = v ? w_st[x] : 0.0f;
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) av[u] = ci[u] >= 0 ? acc[ci[u]] : 0.0f;
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (ci[u] >= 0) acc[ci[u]] = av[u] + sc * wv[u];
                }
            }
            __syncthreads();                       // rows in order; the stage is free again
            if (s_abort) {
                i_abort = i;
                break;
            }
            if (pc.last) {                         // the item's last piece: flush and clear the tile
                const int width = min(P, q.n_post - pc.post0);
                float* gp = q.g + pc.post0;
                if ((width & 3) == 0) {
                    for (int j = 4 * threadIdx.x; j < width; j += 4 * kThreads) {
                        const float4 v = *reinterpret_cast<const float4*>(s_acc + j);
                        if (v.x != 0.f || v.y != 0.f || v.z != 0.f || v.w != 0.f)
                            atomicAdd(reinterpret_cast<float4*>(gp + j), v);
                        *reinterpret_cast<float4*>(s_acc + j) = make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                } else {
                    for (int j = threadIdx.x; j < width; j += kThreads) {
                        if (s_acc[j] != 0.f) atomicAdd(gp + j, s_acc[j]);
                        s_acc[j] = 0.0f;
                    }
                }
                __syncthreads();
            }
        }
        if (i_abort >= 0) {
            // wait (bounded) for the copies still in flight into this CTA's
            // stages: pieces [i_abort, i_abort + kStages) of this batch
            if (threadIdx.x == 0)
                for (int i = i_abort; i < n && i < i_abort + kStages; ++i) {
                    const uint32_t g = used + (uint32_t)i;
                    mbar_wait_bounded(smem_u32(s_full + g % kStages), (g / kStages) & 1u, spin_limit);
                }
            __syncthreads();
            return;
        }
        used += (uint32_t)n;
        __syncthreads();                           // the next batch rewrites the descriptors
    }
}

// Segment form for rows of moderate density (tens to hundreds of synapses of
// a row per 2048-post tile), where one bulk copy and one CTA barrier per
// piece cost more than the piece.  A CTA item is a group of spiking rows (all
// of them, up to kSegRows, when there are enough post spans to give every CTA
// an item) times a span of kSegTiles post tiles: the threads gather the rows'
// segment bounds from the split table into shared memory at once, then each
// warp streams four rows at a time (eight lanes per row, 16-byte loads, four
// in flight per lane) straight into the shared accumulator (shared float
// atomics: the rows of an item hit the same posts), and the span is flushed
// to the conductance with one vector reduction per four posts that received
// events.
constexpr int kSegThreads = 512;
constexpr int kSegTiles = 2;                  // 2048-post tiles per item span (4096 posts, 16 KiB accumulator)
constexpr int kSegRows = 512;                 // rows per item at most

__global__ void __launch_bounds__(kSegThreads) k_propagate_seg(const DevProj* qp, const unsigned long long* ticket,
                                                               int32_t num_tiles) {
    __shared__ float s_acc[kSegTiles * kPostTile];
    __shared__ int64_t s_beg[kSegRows], s_end[kSegRows];
    const DevProj& q = *qp;
    const int slot = (int)((*ticket / (unsigned long long)num_tiles + 1ull) & 1ull);
    const int ns = q.nspk[slot];
    if (ns == 0) return;
    const int nt = q.n_ptiles, P = q.ptile;
    const int n_span = (nt + kSegTiles - 1) / kSegTiles;
    // row groups: as few as give every CTA an item, at most kSegRows rows each
    int64_t groups = ((int64_t)gridDim.x + n_span - 1) / n_span;
    const int64_t min_groups = (ns + kSegRows - 1) / kSegRows;
    if (groups > ns) groups = ns;
    if (groups < min_groups) groups = min_groups;
    const int G = (int)((ns + groups - 1) / groups);
    groups = (ns + G - 1) / G;
    const int64_t items = groups * (int64_t)n_span;
    const float sc = q.scale;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sub = lane >> 3, sl = lane & 7;             // row slot of the warp (4) and lane within it (8)
    constexpr int kSlots = (kSegThreads / 32) * 4;        // rows streamed at once by the CTA
    const int32_t* __restrict__ col = q.col;
    const float* __restrict__ w = q.w;
    for (int j = threadIdx.x; j < kSegTiles * kPostTile; j += kSegThreads) s_acc[j] = 0.0f;
    for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
        const int span = (int)(item % n_span), grp = (int)(item / n_span);
        const int r0 = grp * G, r1 = min(ns, r0 + G);
        const int T0 = span * kSegTiles, T1 = min(nt, T0 + kSegTiles);
        const int post0 = T0 * P;
        for (int r = r0 + (int)threadIdx.x; r < r1; r += kSegThreads) {
            const int64_t* sp = q.split + (int64_t)q.spk[r] * (nt + 1);
            s_beg[r - r0] = sp[T0];
            s_end[r - r0] = sp[T1];
        }
        __syncthreads();                           // bounds ready (and the accumulator clear)
        float* acc = s_acc - post0;
        for (int rr = warp * 4 + sub; rr < r1 - r0; rr += kSlots) {
            const int64_t beg = s_beg[rr], end = s_end[rr];
            // col / w are padded to a multiple of 4 entries: aligned 16-byte
            // loads that start before `end` stay inside the allocation
            for (int64_t k0 = (beg & ~int64_t(3)) + 4 * sl; k0 < end; k0 += 4 * 32) {
                int4 c4[4];
                float4 w4[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int64_t k = k0 + 32 * u;
                    if (k < end) {
                        c4[u] = __ldcs(reinterpret_cast<const int4*>(col + k));
                        w4[u] = __ldcs(reinterpret_cast<const float4*>(w + k));
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int64_t k = k0 + 32 * u;
                    if (k < end) {
                        if (k >= beg) atomicAdd(acc + c4[u].x, sc * w4[u].x);
                        if (k + 1 >= beg && k + 1 < end) atomicAdd(acc + c4[u].y, sc * w4[u].y);
                        if (k + 2 >= beg && k + 2 < end) atomicAdd(acc + c4[u].z, sc * w4[u].z);
                        if (k + 3 >= beg && k + 3 < end) atomicAdd(acc + c4[u].w, sc * w4[u].w);
                    }
                }
            }
        }
        __syncthreads();                           // the span's events are in the accumulator
        const int width = min(kSegTiles * P, q.n_post - post0);
        float* gp = q.g + post0;
        if ((width & 3) == 0) {
            for (int j = 4 * threadIdx.x; j < width; j += 4 * kSegThreads) {
                const float4 v = *reinterpret_cast<const float4*>(s_acc + j);
                if (v.x != 0.f || v.y != 0.f || v.z != 0.f || v.w != 0.f)
                    atomicAdd(reinterpret_cast<float4*>(gp + j), v);
                *reinterpret_cast<float4*>(s_acc + j) = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        } else {
            for (int j = threadIdx.x; j < width; j += kSegThreads) {
                if (s_acc[j] != 0.f) atomicAdd(gp + j, s_acc[j]);
                s_acc[j] = 0.0f;
            }
        }
        // the next item's bounds overwrite s_beg / s_end after every thread
        // has passed this item's second barrier
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

cudaError_t launch_propagate_seg(const DevProj* q, const unsigned long long* ticket, int32_t num_tiles, int sm_count,
                                 cudaStream_t s) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_propagate_seg, kSegThreads, 0);
    if (e != cudaSuccess) return e;
    const int blocks = std::max(1, sm_count * std::max(1, per_sm));
    k_propagate_seg<<<blocks, kSegThreads, 0, s>>>(q, ticket, std::max(1, num_tiles));
    return cudaGetLastError();
}

cudaError_t launch_propagate_tiled(const DevProj* q, int32_t P, const unsigned long long* ticket, int32_t num_tiles,
                                   int sm_count, uint32_t* error, uint32_t spin_limit, cudaStream_t s) {
    const size_t smem = 2 * sizeof(float) * kStages * kChunk + sizeof(Piece) * kMaxPieces + sizeof(float) * (size_t)P +
                        sizeof(unsigned long long) * kStages;
    cudaError_t e = cudaFuncSetAttribute(k_propagate_tiled, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;                        // resident CTAs per SM: one CTA's adds overlap another's copies
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_propagate_tiled, kThreads, smem);
    if (e != cudaSuccess) return e;
    const int blocks = std::max(1, sm_count * std::max(1, per_sm));
    k_propagate_tiled<<<blocks, kThreads, smem, s>>>(q, ticket, std::max(1, num_tiles), error, spin_limit);
    return cudaGetLastError();
}

}  // namespace snn
