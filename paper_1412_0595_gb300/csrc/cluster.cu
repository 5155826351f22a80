// Cluster step engine: a whole small network advanced by one thread-block
// cluster (up to 16 CTAs of 1024 threads on 16 SMs) for many steps per launch.
//
// Each CTA owns a contiguous, warp-aligned slice of the structure-of-arrays
// neurons and keeps their state in registers for the whole launch.  Spikes
// are exchanged through distributed shared memory: every warp writes the
// ballot word of its 32 neurons into a spike bitmask held by every CTA (plain
// remote stores, one writer per word), double-buffered by step parity.  The
// hardware cluster barrier ends the step.  At the start of the next step --
// the model's one-step delay -- each CTA pulls, for every spike of the
// previous step, only the segment of the spiking neuron's row that lands in
// its own slice (segment bounds from a split table built at creation; dense
// rows are sliced directly) into a shared accumulator with local atomics, so
// all 16 SMs share every row and no L2 flag or remote atomic sits on the
// step's critical path.  Spike lists, list lengths and counters are written as
// the other engines write them, so engines can alternate.  Every CTA runs the
// same number of cluster barriers (no early exits).
#include <cooperative_groups.h>

#include "compaction.cuh"
#include "neuron_update.cuh"

namespace cg = cooperative_groups;

namespace snn {

namespace {

constexpr int kCT = 1024;          // threads per CTA
constexpr int kMaxSlicePops = 4 * kCT / kTile + 1;   // populations one CTA's slice can touch
constexpr int kMaxClusterTiles = 16 * 4 * kCT / kTile;  // tiles of the largest network one cluster holds

__device__ __forceinline__ void st_cluster_u64(const unsigned long long* local_addr, int rank, unsigned long long v) {
    const uint32_t laddr = (uint32_t)__cvta_generic_to_shared(local_addr);
    uint32_t raddr;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(raddr) : "r"(laddr), "r"(rank));
    asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(raddr), "l"(v) : "memory");
}

// A spike word: the low 32 bits of the step epoch above the warp's ballot.
// A word whose tag is not the step being read holds no spikes of that step,
// so the words are never cleared.
__device__ __forceinline__ uint32_t word_spikes(unsigned long long w, uint32_t tag) {
    return (uint32_t)(w >> 32) == tag ? (uint32_t)w : 0u;
}

// Adds this CTA's share of the outgoing rows of spiking neuron `idx` (SoA
// index) into the shared accumulators: part `sub` of `parts` (warps) of the
// segment of each row whose post neurons lie in [base, base + per_cta), with
// up to four synapses per lane in flight.
__device__ __forceinline__ void pull_row(const PersistArgs& A, const int32_t* s_tile_pop, const int32_t* s_tile_local,
                                         const int32_t* s_out_begin, int idx, int rank, int n_ranks, int base,
                                         int per_cta, float* acc, int sub, int parts, int lane) {
    const int tile = idx / kTile;
    const int p = s_tile_pop[tile];
    const int local = s_tile_local[tile] + (idx % kTile);
    const int stride = 32 * parts;
    for (int qq = s_out_begin[p]; qq < s_out_begin[p + 1]; ++qq) {
        const DevProj& Q = A.projs[__ldg(A.out_list + qq)];
        const float sc = Q.scale;
        float* mine = acc + Q.channel * per_cta + (Q.post_soa - base);
        if (Q.layout == SNN_LAYOUT_CSR) {
            const int64_t* sp = Q.csplit + (int64_t)local * (n_ranks + 1) + rank;
            const int64_t sb = __ldg(sp), se = __ldg(sp + 1);
            int64_t x = sb + 32 * sub + lane;
            for (; x + 3 * stride < se; x += 4 * stride) {
                int c[4];
                float w[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) { c[u] = __ldg(Q.col + x + u * stride); w[u] = __ldg(Q.w + x + u * stride); }
#pragma unroll
                for (int u = 0; u < 4; ++u) atomicAdd(mine + c[u], sc * w[u]);
            }
            for (; x < se; x += stride) atomicAdd(mine + __ldg(Q.col + x), sc * __ldg(Q.w + x));
        } else {
            const int lo = max(0, base - Q.post_soa);
            const int hi = min(Q.n_post, base + per_cta - Q.post_soa);
            const float* row = Q.w + (int64_t)local * Q.n_post;
            int j = lo + 32 * sub + lane;
            for (; j + 3 * stride < hi; j += 4 * stride) {
                float w[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) w[u] = __ldg(row + j + u * stride);
#pragma unroll
                for (int u = 0; u < 4; ++u) atomicAdd(mine + j + u * stride, sc * w[u]);
            }
            for (; j < hi; j += stride) atomicAdd(mine + j, sc * __ldg(row + j));
        }
    }
}

template <int NPT>
__global__ void __launch_bounds__(kCT, 1) k_step_cluster(const PersistArgs A, int per_cta) {
    extern __shared__ float s_mem[];
    // spike words [2 parities][n_words] (8-byte aligned at the start), then the
    // accumulators [step parity][channel 0/1][per_cta]
    unsigned long long* bits = reinterpret_cast<unsigned long long*>(s_mem);
    const int n_words = A.n.num_tiles * (kTile / 32);
    float* acc = reinterpret_cast<float*>(bits + 2 * n_words);
    __shared__ DevPop s_pops[kMaxSlicePops];
    __shared__ int32_t s_tile_pop[kMaxClusterTiles], s_tile_local[kMaxClusterTiles];
    __shared__ int32_t s_out_begin[kMaxClusterTiles + 1];
    __shared__ uint8_t s_tile_heavy[kMaxClusterTiles];
    __shared__ int32_t s_heavy[32];                        // bitmask words of heavy rows
    __shared__ int32_t s_n_heavy;
    __shared__ unsigned long long s_pop_spikes[kMaxSlicePops];   // spikes of this launch per slice population
    cg::cluster_group cluster = cg::this_cluster();
    const NeuronArgs& a = A.n;
    const int n_ranks = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int base = rank * per_cta;                       // first owned SoA index
    const int n_soa = a.num_tiles * kTile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned long long T0 = *a.ticket;
    const unsigned long long epoch0 = T0 / (unsigned long long)a.num_tiles;
    const unsigned long long ebase = *a.epoch_base;
    const PhiloxKey key{a.seed_lo, a.seed_hi};
    const int last_idx = min(base + per_cta, n_soa) - 1;
    const int p_lo = base < n_soa ? a.tile_pop[base / kTile] : 0;
    const int p_hi = last_idx >= base ? a.tile_pop[last_idx / kTile] : p_lo - 1;
    for (int p = p_lo; p <= p_hi; ++p) copy_pop(s_pops + (p - p_lo), a.pops + p);
    for (int j = threadIdx.x; j < 4 * per_cta; j += kCT) acc[j] = 0.0f;
    for (int j = threadIdx.x; j < 2 * n_words; j += kCT) bits[j] = 0ull;
    for (int p = threadIdx.x; p < kMaxSlicePops; p += kCT) s_pop_spikes[p] = 0ull;
    for (int tl = threadIdx.x; tl < a.num_tiles; tl += kCT) {
        const int p = a.tile_pop[tl];
        s_tile_pop[tl] = p;
        s_tile_local[tl] = (tl - a.pops[p].first_tile) * kTile;
    }
    const int n_pops = a.tile_pop[a.num_tiles - 1] + 1;
    for (int p = threadIdx.x; p <= n_pops; p += kCT) s_out_begin[p] = A.out_begin[p];
    __syncthreads();
    // Heavy rows: populations whose outgoing rows put, on average, 64 or more
    // synapses into one CTA's slice.  Every warp takes a share of each of their
    // spikes; the other spikes go one warp each.  At most 32 words are heavy.
    if (threadIdx.x == 0) {
        int nh = 0;
        for (int tl = 0; tl < a.num_tiles; ++tl) {
            const int p = s_tile_pop[tl];
            const DevPop& P = a.pops[p];
            float work = 0.0f;
            for (int qq = s_out_begin[p]; qq < s_out_begin[p + 1]; ++qq) {
                const DevProj& Q = A.projs[A.out_list[qq]];
                if (Q.layout == SNN_LAYOUT_CSR)
                    work += Q.n_pre > 0 ? (float)Q.row_ptr[Q.n_pre] / ((float)Q.n_pre * n_ranks) : 0.0f;
                else
                    work += (float)Q.n_post / n_ranks;
            }
            const int n_in_tile = min(kTile, P.n - s_tile_local[tl]);
            const int words = (n_in_tile + 31) / 32;
            s_tile_heavy[tl] = work >= 64.0f ? 1 : 0;
            if (work >= 64.0f) {
                for (int j = 0; j < words; ++j)
                    if (nh + j < 32) s_heavy[nh + j] = tl * (kTile / 32) + j;
                nh += words;
            }
        }
        if (nh > 32) {                                     // too many: every spike goes one warp each
            for (int tl = 0; tl < a.num_tiles; ++tl) s_tile_heavy[tl] = 0;
            nh = 0;
        }
        s_n_heavy = nh;
    }

    NeuronState st[NPT];
    int pop_of[NPT], local_of[NPT], n_spk[NPT];
    bool live[NPT];
#pragma unroll
    for (int u = 0; u < NPT; ++u) {
        const int off = threadIdx.x + u * kCT;
        const int idx = base + off;
        live[u] = false;
        pop_of[u] = 0;
        local_of[u] = 0;
        n_spk[u] = 0;
        st[u] = NeuronState{};
        if (off < per_cta && idx < n_soa) {
            const int tile = idx / kTile;
            const int p = a.tile_pop[tile];
            const DevPop& P = a.pops[p];
            const int local = (tile - P.first_tile) * kTile + (idx % kTile);
            if (local < P.n) {
                live[u] = true;
                pop_of[u] = p - p_lo;
                local_of[u] = local;
                if (P.kind != SNN_POP_SOURCE)
                    st[u] = NeuronState{a.V[idx], a.m[idx], a.h[idx], a.n[idx], a.g0[idx], a.g1[idx], a.iext[idx]};
            }
        }
    }
    // the list lengths of the launch's last step (and of the step after it)
    // start at zero; only the last step writes the API spike list
#pragma unroll
    for (int u = 0; u < NPT; ++u)
        if (live[u] && local_of[u] == 0) {
            s_pops[pop_of[u]].nspk[0] = 0;
            s_pops[pop_of[u]].nspk[1] = 0;
        }
    cluster.sync();                                        // words and list lengths cleared everywhere

    for (int k = 0; k <= A.n_steps; ++k) {
        const unsigned long long e64 = epoch0 + (unsigned long long)k;
        const int slot = (int)(e64 & 1ull);
        // the accumulators alternate by step, so a step's clearing and the
        // next-but-one step's adds are ordered by the CTA barrier between them
        float* acc_k = acc + (k & 1) * 2 * per_cta;
        // ---- pull: the previous step's spikes, my slice of their rows --------
        // Light rows: each lane reads one word; the warp then adds, spike by
        // spike, this CTA's segment of each row.  Heavy rows: every warp reads
        // the heavy words and adds a 1/32 share of each segment.
        if (k > 0) {
            const unsigned long long* prev = bits + (slot ^ 1) * n_words;
            const uint32_t tag = (uint32_t)(e64 - 1ull);
            for (int w0 = warp * 32; w0 < n_words; w0 += kCT) {
                const int wd = w0 + lane;
                const uint32_t m = (wd < n_words && !s_tile_heavy[wd / (kTile / 32)]) ? word_spikes(prev[wd], tag) : 0u;
                unsigned nz = __ballot_sync(0xffffffffu, m != 0u);
                while (nz) {
                    const int l = __ffs(nz) - 1;
                    nz &= nz - 1u;
                    uint32_t mm = __shfl_sync(0xffffffffu, m, l);
                    while (mm) {
                        const int bit = __ffs(mm) - 1;
                        mm &= mm - 1u;
                        pull_row(A, s_tile_pop, s_tile_local, s_out_begin, (w0 + l) * 32 + bit, rank, n_ranks, base,
                                 per_cta, acc_k, 0, 1, lane);
                    }
                }
            }
            const int n_heavy = s_n_heavy;
            if (n_heavy > 0) {
                const int hw = lane < n_heavy ? s_heavy[lane] : 0;
                const uint32_t hm = lane < n_heavy ? word_spikes(prev[hw], tag) : 0u;
                unsigned nz = __ballot_sync(0xffffffffu, hm != 0u);
                while (nz) {
                    const int l = __ffs(nz) - 1;
                    nz &= nz - 1u;
                    uint32_t mm = __shfl_sync(0xffffffffu, hm, l);
                    const int wd = __shfl_sync(0xffffffffu, hw, l);
                    while (mm) {
                        const int bit = __ffs(mm) - 1;
                        mm &= mm - 1u;
                        pull_row(A, s_tile_pop, s_tile_local, s_out_begin, wd * 32 + bit, rank, n_ranks, base,
                                 per_cta, acc_k, warp, kCT / 32, lane);
                    }
                }
            }
            __syncthreads();                                // events in acc_k
        }
        if (k == A.n_steps) break;                         // the last pull folds into g below
        const uint32_t t = (uint32_t)(e64 - ebase);
        const bool last = k == A.n_steps - 1;
        unsigned long long* cur = bits + slot * n_words;
        bool wrote = false;                                // this warp stored spike words
#pragma unroll
        for (int u = 0; u < NPT; ++u) {
            const int off = threadIdx.x + u * kCT;
            const int idx = base + off;
            bool spike = false;
            if (live[u]) {
                const DevPop& P = s_pops[pop_of[u]];
                if (P.kind != SNN_POP_SOURCE) {
                    st[u].g0 += acc_k[off];
                    st[u].g1 += acc_k[per_cta + off];
                    acc_k[off] = 0.0f;
                    acc_k[per_cta + off] = 0.0f;
                }
                float isyn;
                spike = neuron_step(P, key, t, local_of[u], a.hs, a.n_sub, st[u], &isyn);
                if (P.kind != SNN_POP_SOURCE) {
                    if (isnan(st[u].V)) atomicAdd(P.nan_count, 1ull);
                    if (a.isyn_rec) a.isyn_rec[idx] = isyn;
                }
                n_spk[u] += spike ? 1 : 0;
            }
            const unsigned ballot = __ballot_sync(0xffffffffu, spike);
            if (ballot && off < per_cta) {
                wrote = true;
                // the warp's 32 neurons are one word of every CTA's spike words
                const int wd = (base + u * kCT + warp * 32) / 32;
                if (lane < n_ranks) st_cluster_u64(cur + wd, lane, ((unsigned long long)(uint32_t)e64 << 32) | ballot);
                // a warp's neurons share one population
                if (lane == 0) atomicAdd(s_pop_spikes + pop_of[u], (unsigned long long)__popc(ballot));
                if (last) {                                // the API spike list of the last step
                    const DevPop& P = s_pops[pop_of[u]];
                    int pos = 0;
                    if (lane == 0) pos = atomicAdd(P.nspk + slot, __popc(ballot));
                    pos = __shfl_sync(0xffffffffu, pos, 0);
                    if (spike) P.spk[pos + __popc(ballot & ((1u << lane) - 1u))] = local_of[u];
                }
            }
        }
        // End of step: only warps that stored spike words need release
        // ordering (a cluster-scope fence); the barrier itself is relaxed and
        // its wait acquires.  Shared accumulators need no cluster ordering
        // (see acc_k above), so a step without spikes runs no fence.
        if (wrote) asm volatile("fence.acq_rel.cluster;" ::: "memory");
        asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
        asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
    }
    const float* acc_end = acc + (A.n_steps & 1) * 2 * per_cta;

    // fold the last step's events (pulled above), write the state and the
    // launch's spike counts back
#pragma unroll
    for (int u = 0; u < NPT; ++u) {
        if (!live[u]) continue;
        const DevPop& P = s_pops[pop_of[u]];
        if (n_spk[u]) P.neuron_spikes[local_of[u]] += n_spk[u];
        if (P.kind == SNN_POP_SOURCE) continue;
        const int off = threadIdx.x + u * kCT;
        const int idx = base + off;
        st[u].g0 += acc_end[off];
        st[u].g1 += acc_end[per_cta + off];
        a.V[idx] = st[u].V; a.m[idx] = st[u].m; a.h[idx] = st[u].h; a.n[idx] = st[u].n;
        a.g0[idx] = st[u].g0; a.g1[idx] = st[u].g1; a.iext[idx] = st[u].ie;
    }
    const int tp = (int)threadIdx.x;                       // signed: an empty slice has p_hi - p_lo = -1
    if (tp <= p_hi - p_lo && s_pop_spikes[tp]) atomicAdd(s_pops[tp].spike_count, s_pop_spikes[tp]);
    cluster.sync();                                        // no CTA leaves while others may read its memory
    if (rank == 0 && threadIdx.x == 0)
        *a.ticket = T0 + (unsigned long long)A.n_steps * (unsigned long long)a.num_tiles;
}

// split[i][r] = first synapse of row i whose post lies in CTA r's slice or later
__global__ void k_cluster_splits(const int64_t* row_ptr, const int32_t* col, int32_t n_pre, int32_t post_soa,
                                 int32_t n_post, int32_t n_ranks, int32_t per_cta, int64_t* split) {
    const int64_t total = (int64_t)n_pre * (n_ranks + 1);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / (n_ranks + 1);
        const int64_t r = e - i * (n_ranks + 1);
        int64_t key = r * per_cta - post_soa;
        key = key < 0 ? 0 : (key > n_post ? n_post : key);
        int64_t lo = row_ptr[i], hi = row_ptr[i + 1];
        while (lo < hi) {
            const int64_t mid = lo + ((hi - lo) >> 1);
            if (col[mid] < key) lo = mid + 1;
            else hi = mid;
        }
        split[e] = lo;
    }
}

size_t cluster_smem(int per_cta, int num_tiles) {
    return sizeof(unsigned long long) * 2 * (size_t)num_tiles * (kTile / 32) + sizeof(float) * 4 * (size_t)per_cta;
}

template <int NPT>
cudaError_t launch_npt(const PersistArgs& a, int cl, int per_cta, cudaStream_t s) {
    const size_t smem = cluster_smem(per_cta, a.n.num_tiles);
    cudaError_t e = cudaFuncSetAttribute(k_step_cluster<NPT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    // always opted in: the kernel's static shared memory counts toward the
    // 48 KiB that a launch may use without the attribute
    e = cudaFuncSetAttribute(k_step_cluster<NPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(cl);
    cfg.blockDim = dim3(kCT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_step_cluster<NPT>, a, per_cta);
}

}  // namespace

// Cluster size and neurons per CTA for a network of n_total (padded) neurons,
// or 0 when it does not fit one cluster (16 CTAs x 1024 threads x 4 neurons).
int cluster_plan(int n_total, int n_pops, int* per_cta) {
    if (n_pops > kMaxClusterTiles) return 0;
    const int warps = (n_total + 31) / 32;
    for (int cl : {16, 8}) {
        const int pc = (warps + cl - 1) / cl * 32;          // whole warps per CTA
        if (pc <= 4 * kCT) {
            *per_cta = pc;
            return cl;
        }
    }
    return 0;
}

cudaError_t cluster_supported(int cl, int per_cta, int num_tiles, bool* ok) {
    *ok = false;
    const size_t smem = cluster_smem(per_cta, num_tiles);
    cudaError_t e = cudaFuncSetAttribute(k_step_cluster<4>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_step_cluster<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(cl);
    cfg.blockDim = dim3(kCT);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    e = cudaOccupancyMaxActiveClusters(&n, k_step_cluster<4>, &cfg);
    if (e != cudaSuccess) return e;
    *ok = n >= 1;
    return cudaSuccess;
}

cudaError_t launch_cluster_splits(const int64_t* row_ptr, const int32_t* col, int32_t n_pre, int32_t post_soa,
                                  int32_t n_post, int32_t n_ranks, int32_t per_cta, int64_t* split, cudaStream_t s) {
    const int64_t total = (int64_t)n_pre * (n_ranks + 1);
    if (total == 0) return cudaSuccess;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 4096);
    k_cluster_splits<<<blocks, 256, 0, s>>>(row_ptr, col, n_pre, post_soa, n_post, n_ranks, per_cta, split);
    return cudaGetLastError();
}

cudaError_t launch_cluster(const PersistArgs& a, int cl, int per_cta, cudaStream_t s) {
    if (a.n.num_tiles == 0 || a.n_steps <= 0) return cudaSuccess;
    const int npt = (per_cta + kCT - 1) / kCT;
    if (npt <= 1) return launch_npt<1>(a, cl, per_cta, s);
    if (npt <= 2) return launch_npt<2>(a, cl, per_cta, s);
    return launch_npt<4>(a, cl, per_cta, s);
}

}  // namespace snn
