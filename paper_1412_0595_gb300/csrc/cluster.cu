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

constexpr int kCT = 1024;          // a CTA's slice holds up to 4 kCT neurons
constexpr int kMaxThreads = 512;   // threads per CTA at most (128 registers a thread)
constexpr int kMaxSlicePops = 4 * kCT / kTile + 1;   // populations one CTA's slice can touch
constexpr int kMaxClusterTiles = 16 * 4 * kCT / kTile;  // tiles of the largest network one cluster holds
constexpr int kMaxClusterProjs = 64;                 // projections of a network the cluster engine runs

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

// What a pull needs of a projection, copied into shared memory at launch
// start so that a spike's row costs one dependent global load (its synapses).
struct ClusterProj {
    const int32_t* col;
    const float* w;
    const int64_t* csplit;     // [n_pre][cluster size + 1] row segments per CTA slice
    int32_t layout, channel, post_soa, n_post;
    float scale;
    int32_t seg_off;           // compressed rows: first row in the shared segment cache, or -1
};

// Adds this CTA's share of the outgoing rows of spiking neuron `local` of
// population p (its outgoing projections are s_out_list[qb .. qe)) into the
// shared accumulators: part `sub` of `parts` (warps) of the segment of each
// row whose post neurons lie in [base, base + per_cta), with up to four
// synapses per lane in flight.
__device__ __forceinline__ void pull_row(const ClusterProj* s_proj, const int32_t* s_out_list,
                                         const longlong2* s_seg, int local, int qb, int qe, int rank,
                                         int n_ranks, int base, int per_cta, float* acc, int sub, int parts, int lane) {
    const int stride = 32 * parts;
    for (int qq = qb; qq < qe; ++qq) {
        const ClusterProj& Q = s_proj[s_out_list[qq]];
        const float sc = Q.scale;
        float* mine = acc + Q.channel * per_cta + (Q.post_soa - base);
        if (Q.layout == SNN_LAYOUT_CSR) {
            int64_t sb, se;
            if (Q.seg_off >= 0) {
                const longlong2 g = s_seg[Q.seg_off + local];
                sb = g.x;
                se = g.y;
            } else {
                const int64_t* sp = Q.csplit + (int64_t)local * (n_ranks + 1) + rank;
                sb = __ldg(sp);
                se = __ldg(sp + 1);
            }
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

template <int PPT, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) k_step_cluster(const PersistArgs A, int per_cta, int n_projs, int seg_rows) {
    extern __shared__ float s_mem[];
    // row segments [seg_rows] (16-byte aligned at the start), spike words
    // [2 parities][n_words], then the accumulators [step parity][channel 0/1][per_cta]
    longlong2* s_seg = reinterpret_cast<longlong2*>(s_mem);
    unsigned long long* bits = reinterpret_cast<unsigned long long*>(s_seg + seg_rows);
    const int n_words = A.n.num_tiles * (kTile / 32);
    float* acc = reinterpret_cast<float*>(bits + 2 * n_words);
    __shared__ ClusterProj s_proj[kMaxClusterProjs];
    __shared__ int32_t s_out_list[kMaxClusterProjs];
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
    const int T = (int)blockDim.x;
    const int n_warps = T / 32;
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
    for (int j = threadIdx.x; j < 4 * per_cta; j += T) acc[j] = 0.0f;
    for (int j = threadIdx.x; j < 2 * n_words; j += T) bits[j] = 0ull;
    for (int p = threadIdx.x; p < kMaxSlicePops; p += T) s_pop_spikes[p] = 0ull;
    for (int tl = threadIdx.x; tl < a.num_tiles; tl += T) {
        const int p = a.tile_pop[tl];
        s_tile_pop[tl] = p;
        s_tile_local[tl] = (tl - a.pops[p].first_tile) * kTile;
    }
    const int n_pops = a.tile_pop[a.num_tiles - 1] + 1;
    for (int p = threadIdx.x; p <= n_pops; p += T) s_out_begin[p] = A.out_begin[p];
    for (int q = threadIdx.x; q < n_projs; q += T) {
        const DevProj& Q = A.projs[q];
        ClusterProj c;
        c.col = Q.col;
        c.w = Q.w;
        c.csplit = Q.csplit;
        c.layout = Q.layout;
        c.channel = Q.channel;
        c.post_soa = Q.post_soa;
        c.n_post = Q.n_post;
        c.scale = Q.scale;
        // compressed rows, in projection order, share the segment cache while it has room
        int off = 0;
        for (int r = 0; r < q; ++r)
            if (A.projs[r].layout == SNN_LAYOUT_CSR) off += A.projs[r].n_pre;
        c.seg_off = (Q.layout == SNN_LAYOUT_CSR && off + Q.n_pre <= seg_rows) ? off : -1;
        s_proj[q] = c;
        s_out_list[q] = A.out_list[q];
    }
    __syncthreads();
    // this CTA's segment of every cached compressed row
    for (int q = 0; q < n_projs; ++q) {
        const ClusterProj& Q = s_proj[q];
        if (Q.seg_off < 0) continue;
        const int n_pre = A.projs[q].n_pre;
        for (int i = threadIdx.x; i < n_pre; i += T) {
            const int64_t* sp = Q.csplit + (int64_t)i * (n_ranks + 1) + rank;
            s_seg[Q.seg_off + i] = make_longlong2(sp[0], sp[1]);
        }
    }
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
            const int words = 2 * ((n_in_tile + 63) / 64);  // both halves of each 64-neuron group
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

    __syncthreads();                                       // heavy words chosen
    // Each lane keeps one heavy word (if any) with the population, the local
    // index of its bit 0 and the outgoing projection range of its neurons:
    // local of bit b = hlocal + 2 b.
    const int n_heavy = s_n_heavy;
    int hword = -1, hlocal = 0, hqb = 0, hqe = 0;
    if (lane < n_heavy) {
        hword = s_heavy[lane];
        const int tl = hword / (kTile / 32);
        const int hp = s_tile_pop[tl];
        hlocal = s_tile_local[tl] + 64 * ((hword >> 1) & 3) + (hword & 1);
        hqb = s_out_begin[hp];
        hqe = s_out_begin[hp + 1];
    }

    NeuronPair st[PPT];
    int pop_of[PPT], local_of[PPT];
    int2 n_spk[PPT];
    unsigned live[PPT];                                    // bit e: neuron local + e exists
#pragma unroll
    for (int u = 0; u < PPT; ++u) {
        const int off = 2 * ((int)threadIdx.x + u * T);
        const int idx = base + off;
        live[u] = 0u;
        pop_of[u] = 0;
        local_of[u] = 0;
        n_spk[u] = make_int2(0, 0);
        st[u] = NeuronPair{};
        if (off < per_cta && idx < n_soa) {
            const int tile = idx / kTile;
            const int p = a.tile_pop[tile];
            const DevPop& P = a.pops[p];
            const int local = (tile - P.first_tile) * kTile + (idx % kTile);
            if (local < P.n) {
                live[u] = local + 1 < P.n ? 3u : 1u;
                pop_of[u] = p - p_lo;
                local_of[u] = local;
                if (P.kind != SNN_POP_SOURCE) {
                    // pairs start at even SoA offsets: 8-byte aligned loads
                    st[u].V = *reinterpret_cast<const float2*>(a.V + idx);
                    st[u].m = *reinterpret_cast<const float2*>(a.m + idx);
                    st[u].h = *reinterpret_cast<const float2*>(a.h + idx);
                    st[u].n = *reinterpret_cast<const float2*>(a.n + idx);
                    st[u].g0 = *reinterpret_cast<const float2*>(a.g0 + idx);
                    st[u].g1 = *reinterpret_cast<const float2*>(a.g1 + idx);
                    st[u].ie = *reinterpret_cast<const float2*>(a.iext + idx);
                }
            }
        }
    }
    // with one pair per thread, an HH pair's population constants stay in
    // registers for the whole launch
    HHPairConsts hc{};
    bool hh_reg = false;
    if (PPT == 1 && live[0]) {
        const DevPop& P = a.pops[pop_of[0] + p_lo];
        hh_reg = P.kind == SNN_POP_HH;
        if (hh_reg) hc = hh_pair_consts(P, a.hs);
    }
    // Such a pair's drive events and first-substep rates of the next step
    // depend on nothing a pull delivers: they are computed while the
    // end-of-step cluster barrier completes.
    RatesT<float2> r_next{};
    unsigned drive_next = 0u;
    if (PPT == 1 && hh_reg) {
        r_next = hh_rates(st[0].V);
        drive_next = hh_drive_pair(hc, key, (uint32_t)(epoch0 - ebase), local_of[0]);
    }
    // the list lengths of the launch's last step (and of the step after it)
    // start at zero; only the last step writes the API spike list
#pragma unroll
    for (int u = 0; u < PPT; ++u)
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
        // the heavy words and adds a 1/n_warps share of each segment.
        if (k > 0) {
            const unsigned long long* prev = bits + (slot ^ 1) * n_words;
            const uint32_t tag = (uint32_t)(e64 - 1ull);
            // heavy words first: one shared load per lane, issued before the
            // light scan's loads so the latencies overlap
            const uint32_t hm = hword >= 0 ? word_spikes(prev[hword], tag) : 0u;
            for (int w0 = warp * 32; w0 < n_words; w0 += T) {
                const int wd = w0 + lane;
                const unsigned long long wv = wd < n_words ? prev[wd] : 0ull;
                const bool heavy = wd < n_words ? s_tile_heavy[wd / (kTile / 32)] != 0 : true;
                const uint32_t m = heavy ? 0u : word_spikes(wv, tag);
                unsigned nz = __ballot_sync(0xffffffffu, m != 0u);
                while (nz) {
                    const int l = __ffs(nz) - 1;
                    nz &= nz - 1u;
                    uint32_t mm = __shfl_sync(0xffffffffu, m, l);
                    const int w = w0 + l;
                    const int tl = w / (kTile / 32);
                    const int p = s_tile_pop[tl];
                    const int lb = s_tile_local[tl] + 64 * ((w >> 1) & 3) + (w & 1);
                    const int qb = s_out_begin[p], qe = s_out_begin[p + 1];
                    while (mm) {
                        const int bit = __ffs(mm) - 1;
                        mm &= mm - 1u;
                        pull_row(s_proj, s_out_list, s_seg, lb + 2 * bit, qb, qe, rank, n_ranks, base, per_cta, acc_k,
                                 0, 1, lane);
                    }
                }
            }
            unsigned nz = __ballot_sync(0xffffffffu, hm != 0u);
            while (nz) {
                const int l = __ffs(nz) - 1;
                nz &= nz - 1u;
                uint32_t mm = __shfl_sync(0xffffffffu, hm, l);
                const int lb = __shfl_sync(0xffffffffu, hlocal, l);
                const int qb = __shfl_sync(0xffffffffu, hqb, l);
                const int qe = __shfl_sync(0xffffffffu, hqe, l);
                while (mm) {
                    const int bit = __ffs(mm) - 1;
                    mm &= mm - 1u;
                    pull_row(s_proj, s_out_list, s_seg, lb + 2 * bit, qb, qe, rank, n_ranks, base, per_cta, acc_k,
                             warp, n_warps, lane);
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
        for (int u = 0; u < PPT; ++u) {
            const int off = 2 * ((int)threadIdx.x + u * T);
            const int idx = base + off;
            unsigned spike = 0u;
            if (live[u]) {
                const DevPop& P = s_pops[pop_of[u]];
                if (P.kind != SNN_POP_SOURCE) {
                    float2* a0 = reinterpret_cast<float2*>(acc_k + off);
                    float2* a1 = reinterpret_cast<float2*>(acc_k + per_cta + off);
                    st[u].g0 = vadd(st[u].g0, *a0);
                    st[u].g1 = vadd(st[u].g1, *a1);
                    *a0 = make_float2(0.0f, 0.0f);
                    *a1 = make_float2(0.0f, 0.0f);
                }
                float2 isyn;
                if (PPT == 1 && hh_reg)
                    spike = hh_step_pair_given(hc, drive_next, r_next, a.n_sub, st[u], &isyn) & live[u];
                else
                    spike = neuron_step_pair(P, key, t, local_of[u], a.hs, a.n_sub, st[u], &isyn) & live[u];
                if (P.kind != SNN_POP_SOURCE) {
                    const int nans = (isnan(st[u].V.x) ? 1 : 0) + ((live[u] & 2u) && isnan(st[u].V.y) ? 1 : 0);
                    if (nans) atomicAdd(P.nan_count, (unsigned long long)nans);
                    if (a.isyn_rec) {
                        a.isyn_rec[idx] = isyn.x;
                        if (live[u] & 2u) a.isyn_rec[idx + 1] = isyn.y;
                    }
                }
                n_spk[u].x += (int)(spike & 1u);
                n_spk[u].y += (int)(spike >> 1);
            }
            const unsigned b0 = __ballot_sync(0xffffffffu, spike & 1u);
            const unsigned b1 = __ballot_sync(0xffffffffu, spike & 2u);
            if ((b0 | b1) && off < per_cta) {
                wrote = true;
                // the warp's 64 neurons are words 2g and 2g + 1 of every CTA's spike words
                const int wd = (base + 2 * (u * T + warp * 32)) / 32;
                const unsigned long long tg = (unsigned long long)(uint32_t)e64 << 32;
                if (lane < n_ranks) {
                    if (b0) st_cluster_u64(cur + wd, lane, tg | b0);
                    if (b1) st_cluster_u64(cur + wd + 1, lane, tg | b1);
                }
                // a warp's neurons share one population
                const int cnt = __popc(b0) + __popc(b1);
                if (lane == 0) atomicAdd(s_pop_spikes + pop_of[u], (unsigned long long)cnt);
                if (last) {                                // the API spike list of the last step
                    const DevPop& P = s_pops[pop_of[u]];
                    int pos = 0;
                    if (lane == 0) pos = atomicAdd(P.nspk + slot, cnt);
                    pos = __shfl_sync(0xffffffffu, pos, 0);
                    const unsigned lt = (1u << lane) - 1u;
                    const int before = pos + __popc(b0 & lt) + __popc(b1 & lt);
                    if (spike & 1u) P.spk[before] = local_of[u];
                    if (spike & 2u) P.spk[before + (int)(spike & 1u)] = local_of[u] + 1;
                }
            }
        }
        // End of step: only warps that stored spike words need release
        // ordering (a cluster-scope fence); the barrier itself is relaxed and
        // its wait acquires.  Shared accumulators need no cluster ordering
        // (see acc_k above), so a step without spikes runs no fence.
        if (wrote) asm volatile("fence.acq_rel.cluster;" ::: "memory");
        asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
        if (PPT == 1 && hh_reg && !last) {
            r_next = hh_rates(st[0].V);
            drive_next = hh_drive_pair(hc, key, t + 1u, local_of[0]);
        }
        asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
    }
    const float* acc_end = acc + (A.n_steps & 1) * 2 * per_cta;

    // fold the last step's events (pulled above), write the state and the
    // launch's spike counts back
#pragma unroll
    for (int u = 0; u < PPT; ++u) {
        if (!live[u]) continue;
        const DevPop& P = s_pops[pop_of[u]];
        if (n_spk[u].x) P.neuron_spikes[local_of[u]] += n_spk[u].x;
        if (n_spk[u].y) P.neuron_spikes[local_of[u] + 1] += n_spk[u].y;
        if (P.kind == SNN_POP_SOURCE) continue;
        const int off = 2 * ((int)threadIdx.x + u * T);
        const int idx = base + off;
        st[u].g0 = vadd(st[u].g0, *reinterpret_cast<const float2*>(acc_end + off));
        st[u].g1 = vadd(st[u].g1, *reinterpret_cast<const float2*>(acc_end + per_cta + off));
        if (!(live[u] & 2u)) {                             // a padding slot (odd population size) stays zero
            st[u].V.y = st[u].m.y = st[u].h.y = st[u].n.y = 0.0f;
            st[u].g0.y = st[u].g1.y = st[u].ie.y = 0.0f;
        }
        *reinterpret_cast<float2*>(a.V + idx) = st[u].V;
        *reinterpret_cast<float2*>(a.m + idx) = st[u].m;
        *reinterpret_cast<float2*>(a.h + idx) = st[u].h;
        *reinterpret_cast<float2*>(a.n + idx) = st[u].n;
        *reinterpret_cast<float2*>(a.g0 + idx) = st[u].g0;
        *reinterpret_cast<float2*>(a.g1 + idx) = st[u].g1;
        *reinterpret_cast<float2*>(a.iext + idx) = st[u].ie;
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

size_t cluster_smem(int per_cta, int num_tiles, int seg_rows) {
    return sizeof(longlong2) * (size_t)seg_rows + sizeof(unsigned long long) * 2 * (size_t)num_tiles * (kTile / 32) +
           sizeof(float) * 4 * (size_t)per_cta;
}

// Threads of a CTA for a slice of per_cta neurons (a multiple of 64), at most
// 512 so that a thread may hold 128 registers: one neuron pair per thread up
// to 1024 neurons, two up to 2048, four above.
int cluster_threads(int per_cta, int* ppt) {
    *ppt = per_cta <= 1024 ? 1 : per_cta <= 2048 ? 2 : 4;
    const int pairs = per_cta / 2;
    return ((pairs + *ppt - 1) / *ppt + 31) / 32 * 32;
}

// The kernel instance for a slice: one pair per thread with at most 384
// threads (up to 168 registers a thread), else at most 512 threads.
const void* cluster_fn(int per_cta, int* threads) {
    int ppt = 1;
    *threads = cluster_threads(per_cta, &ppt);
    if (ppt == 1 && *threads <= 384) return (const void*)k_step_cluster<1, 384>;
    if (ppt == 1) return (const void*)k_step_cluster<1, kMaxThreads>;
    if (ppt == 2) return (const void*)k_step_cluster<2, kMaxThreads>;
    return (const void*)k_step_cluster<4, kMaxThreads>;
}

cudaLaunchConfig_t cluster_config(int cl, int threads, size_t smem, cudaLaunchAttribute* attr, cudaStream_t s) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(cl);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

cudaError_t prepare(const void* fn, size_t smem) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    // always opted in: the kernel's static shared memory counts toward the
    // 48 KiB that a launch may use without the attribute
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

}  // namespace

// Cluster size and neurons per CTA for a network of n_total (padded) neurons,
// or 0 when it does not fit one cluster (16 CTAs x 4096 neurons, at most 64
// projections).
// Slices are whole 64-neuron warp groups (a warp of neuron pairs).
int cluster_plan(int n_total, int n_pops, int n_projs, int* per_cta) {
    if (n_pops > kMaxClusterTiles || n_projs > kMaxClusterProjs) return 0;
    const int groups = (n_total + 63) / 64;
    for (int cl : {16, 8}) {
        const int pc = (groups + cl - 1) / cl * 64;
        if (pc <= 4 * kCT) {
            *per_cta = pc;
            return cl;
        }
    }
    return 0;
}

cudaError_t cluster_supported(int cl, int per_cta, int num_tiles, int seg_rows, bool* ok) {
    *ok = false;
    const size_t smem = cluster_smem(per_cta, num_tiles, seg_rows);
    int threads = 0;
    const void* fn = cluster_fn(per_cta, &threads);
    cudaError_t e = prepare(fn, smem);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cluster_config(cl, threads, smem, attr, nullptr);
    int n = 0;
    e = cudaOccupancyMaxActiveClusters(&n, fn, &cfg);
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

cudaError_t launch_cluster(const PersistArgs& a, int cl, int per_cta, int n_projs, int seg_rows, cudaStream_t s) {
    if (a.n.num_tiles == 0 || a.n_steps <= 0) return cudaSuccess;
    const size_t smem = cluster_smem(per_cta, a.n.num_tiles, seg_rows);
    int threads = 0;
    const void* fn = cluster_fn(per_cta, &threads);
    cudaError_t e = prepare(fn, smem);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cluster_config(cl, threads, smem, attr, s);
    void* args[] = {const_cast<PersistArgs*>(&a), &per_cta, &n_projs, &seg_rows};
    return cudaLaunchKernelExC(&cfg, fn, args);
}

}  // namespace snn
