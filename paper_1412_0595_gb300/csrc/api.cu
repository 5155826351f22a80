// Host side of the C-ABI (include/snn.h): argument checking, the
// structure-of-arrays layout in HBM, the conductance scaling law, CUDA-graph
// capture of the step loop, and state access.  No exception crosses the ABI.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "snn_internal.cuh"

namespace snn {

namespace {
thread_local std::string g_err;
}  // namespace

snn_status fail(snn_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

snn_status cuda_fail(cudaError_t e, const char* what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return SNN_ERR_CUDA;
}

void* Alloc::get(size_t bytes) {
    bytes = std::max<size_t>(256, (bytes + 255) & ~size_t(255));
    if (have) return a.alloc(bytes, stream, a.ctx);
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return p;
}

void Alloc::put(void* p) {
    if (!p) return;
    if (have) a.free(p, stream, a.ctx);
    else cudaFree(p);
}

}  // namespace snn

namespace snn {

// The step's spike lists of the pre populations of a shared dense projection,
// gathered as one list per instance (spk_off[B + 1], spk) for the batched
// delivery: one CTA scans the list lengths, then its warps copy the lists.
__global__ void __launch_bounds__(1024) k_shared_spike_lists(const int32_t* pre_pop, const int32_t* pre_off, int32_t B,
                                                             const int32_t* nspk, const int32_t* spk_all,
                                                             const unsigned long long* ticket, int32_t num_tiles,
                                                             int32_t* spk_off, int32_t* spk_out) {
    __shared__ int32_t s_w[32];
    __shared__ int32_t s_run;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // list-length slot of the step whose spikes are delivered
    const int slot = (int)((*ticket / (unsigned long long)num_tiles + 1ull) & 1ull);
    if (threadIdx.x == 0) s_run = 0;
    __syncthreads();
    for (int b0 = 0; b0 < B; b0 += 1024) {
        const int b = b0 + (int)threadIdx.x;
        const int c = b < B ? nspk[2 * pre_pop[b] + slot] : 0;
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_w[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const int v = s_w[lane];
            int wi = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += y;
            }
            s_w[lane] = wi - v;
        }
        __syncthreads();
        const int excl = s_run + s_w[warp] + incl - c;
        if (b < B) spk_off[b] = excl;
        __syncthreads();
        if (threadIdx.x == 1023) s_run = excl + c;
        __syncthreads();
    }
    if (threadIdx.x == 0) spk_off[B] = s_run;
    __syncthreads();                                   // the offsets are visible to the whole CTA
    for (int b = warp; b < B; b += 32) {
        const int o = spk_off[b], c = spk_off[b + 1] - o;
        const int32_t* src = spk_all + pre_off[b];
        for (int j = lane; j < c; j += 32) spk_out[o + j] = src[j];
    }
}

}  // namespace snn

using namespace snn;

namespace {

#define CK(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

template <typename T>
snn_status dalloc(snn_net* net, T** out, size_t count, const char* what) {
    void* p = net->mem.get(count * sizeof(T));
    if (!p) return fail(SNN_ERR_OOM, std::string("device allocation failed: ") + what);
    net->owned.push_back(p);
    *out = static_cast<T*>(p);
    return SNN_OK;
}

#define TRY(x)                        \
    do {                              \
        snn_status s_ = (x);          \
        if (s_ != SNN_OK) return s_;  \
    } while (0)

void release(snn_net* net) {
    if (net->graph) cudaGraphExecDestroy(net->graph);
    net->graph = nullptr;
    if (net->cap_stream) cudaStreamDestroy(net->cap_stream);
    net->cap_stream = nullptr;
    for (void* p : net->owned) net->mem.put(p);
    net->owned.clear();
}

struct Guard {   // frees the device allocations of a half-built network
    snn_net* net;
    ~Guard() {
        if (net) {
            release(net);
            delete net;
        }
    }
};

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

snn_status check_pop(const snn_pop_desc& d, int k) {
    const std::string at = "population " + std::to_string(k) + ": ";
    if (d.kind != SNN_POP_HH && d.kind != SNN_POP_SOURCE && d.kind != SNN_POP_IZH)
        return fail(SNN_ERR_INVALID_ARG, at + "bad kind");
    if (d.n < 0 || d.n >= (1 << 30)) return fail(SNN_ERR_INVALID_ARG, at + "n out of range");
    if (d.kind == SNN_POP_HH) {
        if (!finite_pos(d.C)) return fail(SNN_ERR_INVALID_ARG, at + "C must be > 0");
        const double v[] = {d.gNa, d.ENa, d.gK, d.EK, d.gL, d.EL, d.E_syn[0], d.E_syn[1], d.v_thresh,
                            d.drive_amp};
        for (double x : v)
            if (!std::isfinite(x)) return fail(SNN_ERR_INVALID_ARG, at + "non-finite parameter");
        if (d.drive_rate_hz < 0 || !std::isfinite(d.drive_rate_hz))
            return fail(SNN_ERR_INVALID_ARG, at + "drive rate must be >= 0");
    } else if (d.kind == SNN_POP_IZH) {
        for (double x : d.izh)
            if (!std::isfinite(x)) return fail(SNN_ERR_INVALID_ARG, at + "non-finite Izhikevich parameter");
        if (!std::isfinite(d.noise_sigma) || d.noise_sigma < 0 || !std::isfinite(d.bias) || !std::isfinite(d.v_thresh))
            return fail(SNN_ERR_INVALID_ARG, at + "bad Izhikevich input or threshold");
    } else if (d.src_rate_hz < 0 || !std::isfinite(d.src_rate_hz)) {
        return fail(SNN_ERR_INVALID_ARG, at + "source rate must be >= 0");
    }
    return SNN_OK;
}

// Scaling law of Sec. 5.1: s = (k1 / (k2 + nConn) + k3) * c.
snn_status proj_scale(const snn_proj_desc& d, int32_t n_pre, int q, float* out) {
    const double n_conn = d.n_conn > 0.0 ? d.n_conn : d.density * (double)n_pre;
    const double den = d.k2 + n_conn;
    if (!(den > 0.0) || !std::isfinite(den))
        return fail(SNN_ERR_GSCALE, "projection " + std::to_string(q) + ": nConn + k2 <= 0, gScale undefined");
    const double s = (d.k1 / den + d.k3) * d.user_scale;
    if (!std::isfinite(s)) return fail(SNN_ERR_GSCALE, "projection " + std::to_string(q) + ": non-finite scale");
    *out = (float)s;
    return SNN_OK;
}

snn_status sticky(snn_net* net, cudaStream_t s) {
    uint32_t err = 0;
    CK(cudaMemcpyAsync(&err, net->error, sizeof(err), cudaMemcpyDeviceToHost, s), "read error word");
    CK(cudaStreamSynchronize(s), "synchronize");
    if (err & kDevErrTimeout) return fail(SNN_ERR_TIMEOUT, "a bounded device-side wait ran out");
    if (err & kDevErrCsr) return fail(SNN_ERR_CSR, "malformed compressed rows found on the device");
    return SNN_OK;
}

snn_status upload_projs(snn_net* net) {
    std::vector<DevProj> dp(net->projs.size());
    for (size_t q = 0; q < net->projs.size(); ++q) {
        const ProjHost& P = net->projs[q];
        const PopHost& pre = net->pops[P.d.pre];
        const PopHost& post = net->pops[P.d.post];
        DevProj& d = dp[q];
        d.layout = P.d.layout;
        d.n_pre = pre.d.n;
        d.n_post = post.d.n;
        if (P.d.layout == SNN_LAYOUT_CSR)
            d.chunks = std::max<int32_t>(1, (P.max_row + net->chunk - 1) / net->chunk);
        else
            d.chunks = std::max<int32_t>(1, (post.d.n + dense_posts_per_item() - 1) / dense_posts_per_item());
        d.scale = P.scale;
        d.row_ptr = P.row_ptr;
        d.col = P.col;
        d.w = P.w;
        d.g = (P.d.channel == 0 ? net->g0 : net->g1) + post.offset;
        d.spk = net->spk + pre.offset;
        d.nspk = net->nspk + 2 * P.d.pre;
        d.pre_count = net->nrn_count + pre.offset;
        d.acc = net->acc + (P.d.channel == 0 ? 0 : 2 * (size_t)std::max(1, net->n_total)) + post.offset;
        d.post_soa = post.offset;
        d.channel = P.d.channel;
        d.mode = P.mode;
        d.ptile = kPostTile;
        d.n_ptiles = (post.d.n + kPostTile - 1) / kPostTile;
        d.split = P.split;
        d.csplit = P.csplit;
    }
    if (!dp.empty())
        CK(cudaMemcpy(net->d_projs, dp.data(), dp.size() * sizeof(DevProj), cudaMemcpyHostToDevice),
           "upload projection descriptors");
    return SNN_OK;
}

NeuronArgs neuron_args(snn_net* net) {
    NeuronArgs a{};
    a.pops = net->d_pops;
    a.tile_pop = net->tile_pop;
    a.V = net->V; a.m = net->m; a.h = net->h; a.n = net->n;
    a.g0 = net->g0; a.g1 = net->g1; a.iext = net->iext;
    a.isyn_rec = net->record_isyn ? net->isyn : nullptr;
    a.ticket = net->ticket;
    a.epoch_base = net->ticket + 1;
    a.error = net->error;
    a.num_tiles = net->num_tiles;
    a.n_sub = net->n_sub;
    a.hs = (float)(net->dt / net->n_sub);
    a.spin_limit = net->spin_limit;
    a.seed_lo = (uint32_t)net->seed;
    a.seed_hi = (uint32_t)(net->seed >> 32);
    return a;
}

int prop_blocks(snn_net* net) { return net->prop_blocks > 0 ? net->prop_blocks : net->sm_count * 4; }

// Post-tiled propagation pays off when a row has many synapses in each post
// tile and the post population spans at least eight tiles; below that the
// row kernel's global reductions stay in L2 and cost less than the staging.
// Measured crossovers (100 spiking rows, caches flushed; bench_profiles.py
// --tiled-crossover), by synapses of a row per 2048-post tile: on 524,288
// posts and more, segments from 16 (p = 0.01 .. 0.2 at 1,000,000 posts:
// 16-66 us against 18-76 us for the better of the other two), bulk-copied
// pieces from 800 (p = 0.5: 86 against 143 us); on 131,072 to 524,287 posts
// segments from 96 (p = 0.05 at 300,000 posts: 20.5 against 24.6 us) and
// pieces from 300; below, pieces from 256.
// Mode of a compressed-row projection's propagation in the plain engine:
// 0 row kernel, 1 post-tiled through bulk copies, 2 post-tiled segments
// streamed by warps into the shared accumulator.
int32_t tiled_mode(const snn_net* net, const ProjHost& P) {
    if (P.d.layout != SNN_LAYOUT_CSR || net->tiled == 0) return 0;
    if (net->tiled == 1) return 1;
    if (net->tiled == 3) return 2;
    const int32_t n_pre = net->pops[P.d.pre].d.n, n_post = net->pops[P.d.post].d.n;
    if (n_post < 8 * kPostTile || n_pre == 0) return 0;
    const double per_tile = (double)P.nnz / n_pre * kPostTile / n_post;
    if (n_post >= 256 * kPostTile) return per_tile >= 800.0 ? 1 : per_tile >= 16.0 ? 2 : 0;
    if (n_post >= 64 * kPostTile) return per_tile >= 300.0 ? 1 : per_tile >= 96.0 ? 2 : 0;
    return per_tile >= 256.0 ? 1 : 0;
}

}  // namespace

// The propagation mode of every projection under the SNN_OPT_TILED value `tiled`.
std::vector<int32_t> snn::propagation_modes(const snn_net* net, int32_t tiled) {
    snn_net probe_opts;
    probe_opts.tiled = tiled;
    probe_opts.pops = net->pops;
    std::vector<int32_t> m;
    for (const auto& P : net->projs) m.push_back(tiled_mode(&probe_opts, P));
    return m;
}

namespace {

snn_status setup_tiled(snn_net* net, cudaStream_t s) {
    for (auto& P : net->projs) {
        P.mode = tiled_mode(net, P);
        if (P.mode != 0 && !P.split) {
            const int32_t n_pre = net->pops[P.d.pre].d.n, n_post = net->pops[P.d.post].d.n;
            const int32_t nt = (n_post + kPostTile - 1) / kPostTile;
            TRY(dalloc(net, &P.split, (size_t)n_pre * (nt + 1) + 1, "row splits"));
            CK(launch_row_splits(P.row_ptr, P.col, n_pre, nt, kPostTile, P.split, s), "row splits");
        }
    }
    CK(cudaStreamSynchronize(s), "synchronize");
    return upload_projs(net);
}

// Propagation of the projections in `dev` (n of them, host copies in `host`).
cudaError_t launch_projections(snn_net* net, const DevProj* dev, const ProjHost* const* host, int n, cudaStream_t s) {
    PropArgs p{dev, n, net->chunk, net->ticket, std::max(1, net->num_tiles)};
    // the row kernel only when some projection takes it (it would find no items otherwise)
    bool rows = false;
    for (int q = 0; q < n; ++q) rows = rows || host[q]->mode == 0;
    cudaError_t e = rows ? launch_propagate(p, prop_blocks(net), s) : cudaSuccess;
    for (int q = 0; q < n && e == cudaSuccess; ++q)
        if (host[q]->mode == 1)
            e = launch_propagate_tiled(dev + q, kPostTile, net->ticket, std::max(1, net->num_tiles), net->sm_count,
                                       net->error, net->spin_limit, s);
        else if (host[q]->mode == 2)
            e = launch_propagate_seg(dev + q, net->ticket, std::max(1, net->num_tiles), net->sm_count, s);
    return e;
}

cudaError_t launch_all_projections(snn_net* net, cudaStream_t s) {
    if (net->projs.empty()) return cudaSuccess;
    std::vector<const ProjHost*> host;
    for (const auto& P : net->projs) host.push_back(&P);
    return launch_projections(net, net->d_projs, host.data(), (int)host.size(), s);
}

bool use_cluster(const snn_net* net) {
    if (net->cluster_size == 0 || !net->shared.empty()) return false;
    return net->engine == 3 || net->engine == 2;
}

bool use_persistent(const snn_net* net) {
    if (!net->shared.empty()) return false;      // shared dense projections: the plain engine's step
    if (net->engine == 1) return net->persist_grid > 0;
    if (net->engine != 2) return false;
    return net->num_tiles > 0 && net->num_tiles <= net->persist_grid;   // one resident CTA per tile
}

PersistArgs persist_args(snn_net* net, int32_t n_steps) {
    PersistArgs p{};
    p.n = neuron_args(net);
    p.projs = net->d_projs;
    p.out_begin = net->out_begin;
    p.out_list = net->out_list;
    const size_t NT = std::max<size_t>(1, (size_t)net->n_total);
    p.acc0 = net->acc;
    p.acc1 = net->acc + 2 * NT;
    p.acc_stride = (int32_t)NT;
    p.n_steps = n_steps;
    p.barrier_extra = net->barrier_extra;
    p.bar = net->bar;
    return p;
}

cudaError_t enqueue_persistent(snn_net* net, int64_t n_steps, cudaStream_t s) {
    while (n_steps > 0) {
        const int32_t k = (int32_t)std::min<int64_t>(n_steps, net->persist_steps);
        cudaError_t e = launch_persistent(persist_args(net, k), net->persist_grid, s);
        if (e != cudaSuccess) return e;
        n_steps -= k;
    }
    return cudaSuccess;
}

cudaError_t launch_shared_dense(snn_net* net, cudaStream_t s) {
    for (const SharedDense& d : net->shared) {
        k_shared_spike_lists<<<1, 1024, 0, s>>>(d.pre_pop, d.pre_off, d.B, net->nspk, net->spk, net->ticket,
                                                std::max(1, net->num_tiles), d.spk_off, d.spk);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const int64_t thr = (int64_t)std::ceil(net->shared_density * (double)d.B * d.n_pre);
        e = dense_batch_launch(d.h, d.B, d.spk_off, d.spk, d.scale, d.G, d.ldg, net->shared_engine,
                               std::max<int64_t>(1, thr), s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t enqueue_step(snn_net* net, cudaStream_t s) {
    cudaError_t e = launch_neuron_step(neuron_args(net), s);
    if (e != cudaSuccess) return e;
    e = launch_all_projections(net, s);
    if (e != cudaSuccess || net->shared.empty()) return e;
    return launch_shared_dense(net, s);
}

void drop_graph(snn_net* net) {
    if (net->graph) cudaGraphExecDestroy(net->graph);
    net->graph = nullptr;
    net->graph_len = 0;
}

snn_status ensure_graph(snn_net* net) {
    if (net->graph && net->graph_len == net->graph_steps) return SNN_OK;
    drop_graph(net);
    if (!net->cap_stream) CK(cudaStreamCreateWithFlags(&net->cap_stream, cudaStreamNonBlocking), "create stream");
    CK(cudaStreamBeginCapture(net->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    cudaError_t e = cudaSuccess;
    for (int64_t k = 0; k < net->graph_steps && e == cudaSuccess; ++k) e = enqueue_step(net, net->cap_stream);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(net->cap_stream, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(e, "capture step");
    }
    if (e2 != cudaSuccess) return cuda_fail(e2, "end capture");
    e = cudaGraphInstantiate(&net->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "instantiate graph");
    net->graph_len = net->graph_steps;
    return SNN_OK;
}

float* field_base(snn_net* net, int32_t field) {
    switch (field) {
    case SNN_FIELD_V: return net->V;
    case SNN_FIELD_M: return net->m;
    case SNN_FIELD_H: return net->h;
    case SNN_FIELD_N: return net->n;
    case SNN_FIELD_G0: return net->g0;
    case SNN_FIELD_G1: return net->g1;
    case SNN_FIELD_IEXT: return net->iext;
    case SNN_FIELD_ISYN: return net->isyn;
    default: return nullptr;
    }
}

snn_status create_impl(const snn_pop_desc* pops, int32_t n_pops, const snn_proj_desc* projs, int32_t n_projs,
                       double dt, int32_t n_sub, uint64_t seed, const std::vector<uint32_t>& tags,
                       const snn_allocator* alloc, cudaStream_t s, snn_net** out) {
    if (!out) return fail(SNN_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!pops || n_pops < 1 || n_pops > kMaxPops) return fail(SNN_ERR_INVALID_ARG, "need 1..4096 populations");
    if (n_projs < 0 || n_projs > kMaxProjs || (n_projs > 0 && !projs))
        return fail(SNN_ERR_INVALID_ARG, "need 0..4096 projections");
    if (!finite_pos(dt)) return fail(SNN_ERR_INVALID_ARG, "dt must be > 0");
    if (n_sub < 1 || n_sub > 1024) return fail(SNN_ERR_INVALID_ARG, "n_substeps must be in 1..1024");
    if (alloc && (!alloc->alloc || !alloc->free)) return fail(SNN_ERR_INVALID_ARG, "allocator without alloc/free");
    for (int k = 0; k < n_pops; ++k) TRY(check_pop(pops[k], k));
    std::vector<float> scales((size_t)n_projs);
    for (int q = 0; q < n_projs; ++q) {
        const snn_proj_desc& d = projs[q];
        const std::string at = "projection " + std::to_string(q) + ": ";
        if (d.pre < 0 || d.pre >= n_pops || d.post < 0 || d.post >= n_pops)
            return fail(SNN_ERR_INVALID_ARG, at + "pre/post out of range");
        if (pops[d.post].kind == SNN_POP_SOURCE) return fail(SNN_ERR_INVALID_ARG, at + "post must not be a source");
        if (d.synapse == SNN_SYN_GRADED && pops[d.post].kind != SNN_POP_HH)
            return fail(SNN_ERR_INVALID_ARG, at + "graded synapses target HH populations");
        if (d.channel != 0 && d.channel != 1) return fail(SNN_ERR_INVALID_ARG, at + "channel must be 0 or 1");
        if (d.layout != SNN_LAYOUT_CSR && d.layout != SNN_LAYOUT_DENSE)
            return fail(SNN_ERR_INVALID_ARG, at + "bad layout");
        if (d.synapse != SNN_SYN_EXP && d.synapse != SNN_SYN_GRADED) return fail(SNN_ERR_INVALID_ARG, at + "bad synapse kind");
        if ((d.synapse == SNN_SYN_GRADED) != graded_requested(projs, n_projs))
            return fail(SNN_ERR_INVALID_ARG, at + "a network is either spiking (exponential) or graded throughout");
        if (d.input_dense) {
            if (d.layout != SNN_LAYOUT_DENSE) return fail(SNN_ERR_INVALID_ARG, at + "dense input needs dense layout");
            if (!d.w && (int64_t)pops[d.pre].n * pops[d.post].n > 0) return fail(SNN_ERR_INVALID_ARG, at + "w is NULL");
        } else {
            if (!d.row_ptr) return fail(SNN_ERR_INVALID_ARG, at + "row_ptr is NULL");
            if (d.nnz < 0 || d.nnz >= (int64_t(1) << 40)) return fail(SNN_ERR_INVALID_ARG, at + "bad nnz");
            if (d.nnz > 0 && (!d.col || !d.w)) return fail(SNN_ERR_INVALID_ARG, at + "col/w is NULL");
        }
        if (!std::isfinite(d.user_scale)) return fail(SNN_ERR_INVALID_ARG, at + "non-finite user scale");
        TRY(proj_scale(d, pops[d.pre].n, q, &scales[q]));
    }

    snn_net* net = new snn_net();
    Guard guard{net};
    if (alloc) {
        net->mem.a = *alloc;
        net->mem.have = true;
    }
    net->mem.stream = s;
    net->dt = dt;
    net->n_sub = n_sub;
    net->seed = seed;
    int dev = 0;
    CK(cudaGetDevice(&dev), "get device");
    CK(cudaDeviceGetAttribute(&net->sm_count, cudaDevAttrMultiProcessorCount, dev), "SM count");
    {
        int l2 = 0;
        CK(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev), "L2 size");
        net->l2_bytes = l2;
    }

    // ---- structure-of-arrays layout: populations padded to whole tiles ----
    int64_t off = 0, tiles = 0;
    net->pops.resize((size_t)n_pops);
    for (int k = 0; k < n_pops; ++k) {
        PopHost& P = net->pops[k];
        P.d = pops[k];
        P.offset = (int32_t)off;
        P.first_tile = (int32_t)tiles;
        P.n_tiles = (P.d.n + kTile - 1) / kTile;
        off += (int64_t)P.n_tiles * kTile;
        tiles += P.n_tiles;
        if (off >= (int64_t(1) << 31)) return fail(SNN_ERR_INVALID_ARG, "too many neurons in total");
    }
    net->n_total = (int32_t)off;
    net->num_tiles = (int32_t)tiles;
    const size_t NT = std::max<size_t>(1, (size_t)net->n_total);

    float* state = nullptr;
    TRY(dalloc(net, &state, 8 * NT, "state"));
    net->V = state; net->m = state + NT; net->h = state + 2 * NT; net->n = state + 3 * NT;
    net->g0 = state + 4 * NT; net->g1 = state + 5 * NT; net->iext = state + 6 * NT; net->isyn = state + 7 * NT;
    TRY(dalloc(net, &net->init_state, 7 * NT, "initial state"));
    TRY(dalloc(net, &net->spk, NT, "spike lists"));
    TRY(dalloc(net, &net->nrn_count, NT, "per-neuron spike counts"));
    TRY(dalloc(net, &net->d_events, 1, "event counter"));
    TRY(dalloc(net, &net->acc, 4 * NT, "event accumulators"));
    TRY(dalloc(net, &net->bar, 1, "grid barrier"));
    TRY(dalloc(net, &net->out_begin, (size_t)n_pops + 1, "outgoing projection offsets"));
    TRY(dalloc(net, &net->out_list, std::max<size_t>(1, (size_t)n_projs), "outgoing projections"));
    CK(cudaMemsetAsync(net->acc, 0, 4 * NT * sizeof(float), s), "clear");
    CK(cudaMemsetAsync(net->bar, 0, sizeof(GridBarrier), s), "clear");
    CK(cudaMemsetAsync(net->nrn_count, 0, NT * sizeof(int32_t), s), "clear");
    TRY(dalloc(net, &net->nspk, 2 * (size_t)n_pops, "spike list lengths"));
    TRY(dalloc(net, &net->counters, 2 * (size_t)n_pops, "counters"));
    TRY(dalloc(net, &net->ticket, 2, "ticket"));
    TRY(dalloc(net, &net->tile_pop, std::max<size_t>(1, (size_t)tiles), "tile map"));
    TRY(dalloc(net, &net->error, 1, "error word"));
    TRY(dalloc(net, &net->d_pops, (size_t)n_pops, "population descriptors"));
    TRY(dalloc(net, &net->d_projs, std::max<size_t>(1, (size_t)n_projs), "projection descriptors"));
    TRY(dalloc(net, &net->d_dbg_proj, 1, "debug descriptor"));
    CK(cudaMemsetAsync(state, 0, 8 * NT * sizeof(float), s), "clear state");
    CK(cudaMemsetAsync(net->nspk, 0, sizeof(int32_t) * 2 * n_pops, s), "clear");
    CK(cudaMemsetAsync(net->counters, 0, sizeof(unsigned long long) * 2 * n_pops, s), "clear");
    CK(cudaMemsetAsync(net->ticket, 0, 2 * sizeof(unsigned long long), s), "clear");
    CK(cudaMemsetAsync(net->error, 0, sizeof(uint32_t), s), "clear");

    // ---- initial potentials, population descriptors, tile map ----
    std::vector<float> v0(NT, 0.0f);
    std::vector<int32_t> tile_pop(std::max<size_t>(1, (size_t)tiles), 0);
    std::vector<DevPop> dp((size_t)n_pops);
    const double hs = dt / n_sub;
    for (int k = 0; k < n_pops; ++k) {
        const PopHost& P = net->pops[k];
        const snn_pop_desc& d = P.d;
        if (d.kind != SNN_POP_SOURCE) {
            if (d.v0 && !d.v0_on_device) std::memcpy(&v0[P.offset], d.v0, sizeof(float) * d.n);
            else std::fill(v0.begin() + P.offset, v0.begin() + P.offset + d.n, (float)d.EL);
        }
        for (int t = 0; t < P.n_tiles; ++t) tile_pop[P.first_tile + t] = k;
        DevPop& q = dp[k];
        q.kind = d.kind;
        q.n = d.n;
        q.offset = P.offset;
        q.first_tile = P.first_tile;
        q.n_tiles = P.n_tiles;
        q.tag = tags[k];
        q.gNa = (float)d.gNa; q.ENa = (float)d.ENa; q.gK = (float)d.gK; q.EK = (float)d.EK;
        q.gL = (float)d.gL; q.EL = (float)d.EL;
        q.hs_over_C = d.kind == SNN_POP_HH ? (float)(hs / d.C) : 0.0f;
        q.E0 = (float)d.E_syn[0]; q.E1 = (float)d.E_syn[1];
        q.d0 = d.tau_syn[0] > 0 ? (float)std::exp(-dt / d.tau_syn[0]) : 0.0f;
        q.d1 = d.tau_syn[1] > 0 ? (float)std::exp(-dt / d.tau_syn[1]) : 0.0f;
        q.v_thresh = (float)d.v_thresh;
        q.drive_amp = (float)d.drive_amp;
        q.drive_dec = d.drive_tau > 0 ? (float)std::exp(-dt / d.drive_tau) : 0.0f;
        q.thr_src = d.kind == SNN_POP_SOURCE ? bernoulli_threshold(d.src_rate_hz * dt * 1e-3) : 0ull;
        q.thr_drive = d.kind == SNN_POP_HH ? bernoulli_threshold(d.drive_rate_hz * dt * 1e-3) : 0ull;
        q.spk = net->spk + P.offset;
        q.nspk = net->nspk + 2 * k;
        q.spike_count = net->counters + 2 * k;
        q.nan_count = net->counters + 2 * k + 1;
        q.neuron_spikes = net->nrn_count + P.offset;
        for (int j = 0; j < 8; ++j) q.izh[j] = (float)d.izh[j];
        q.noise = (float)d.noise_sigma;
        q.bias = (float)d.bias;
        q.dt = (float)dt;
        // channel 1 and the drive current stay zero unless a projection
        // targets the channel or the population is driven (or a caller
        // writes them, see snn_write_state / snn_load_state)
        q.g1_live = 0;
        for (int j = 0; j < n_projs; ++j)
            if (projs[j].post == k && projs[j].channel == 1) q.g1_live = 1;
        q.iext_live = q.thr_drive != 0ull ? 1 : 0;
    }
    CK(cudaMemcpyAsync(net->V, v0.data(), NT * sizeof(float), cudaMemcpyHostToDevice, s), "upload V0");
    for (int k = 0; k < n_pops; ++k) {
        const PopHost& P = net->pops[k];
        if (P.d.kind != SNN_POP_SOURCE && P.d.v0 && P.d.v0_on_device && P.d.n > 0)
            CK(cudaMemcpyAsync(net->V + P.offset, P.d.v0, sizeof(float) * P.d.n, cudaMemcpyDeviceToDevice, s),
               "copy V0");
    }
    CK(cudaMemcpyAsync(net->tile_pop, tile_pop.data(), tile_pop.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s),
       "upload tile map");
    CK(cudaMemcpyAsync(net->d_pops, dp.data(), dp.size() * sizeof(DevPop), cudaMemcpyHostToDevice, s),
       "upload population descriptors");
    CK(launch_init_state(net->d_pops, n_pops, net->tile_pop, net->num_tiles, net->V, net->m, net->h, net->n,
                         net->g0, net->g1, net->iext, seed, s),
       "initialise state");

    // ---- projections: copy, validate, measure ----
    net->projs.resize((size_t)n_projs);
    std::vector<int32_t*> max_rows;
    int32_t* d_max = nullptr;
    if (n_projs > 0) {
        TRY(dalloc(net, &d_max, (size_t)n_projs, "row maxima"));
        CK(cudaMemsetAsync(d_max, 0, sizeof(int32_t) * n_projs, s), "clear");
    }
    for (int q = 0; q < n_projs; ++q) {
        ProjHost& P = net->projs[q];
        P.d = projs[q];
        P.scale = scales[q];
        const int32_t n_pre = pops[P.d.pre].n, n_post = pops[P.d.post].n;
        const cudaMemcpyKind kind = P.d.on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        if (P.d.input_dense) {
            const int64_t cnt = (int64_t)n_pre * n_post;
            P.nnz = cnt;
            TRY(dalloc(net, &P.w, (size_t)cnt + 4, "dense weights"));
            if (cnt > 0) CK(cudaMemcpyAsync(P.w, P.d.w, sizeof(float) * cnt, kind, s), "copy weights");
            continue;
        }
        P.nnz = P.d.nnz;
        const size_t padded = (size_t)((P.nnz + 3) / 4 * 4 + 4);
        int64_t* rp = nullptr;
        int32_t* col = nullptr;
        float* w = nullptr;
        TRY(dalloc(net, &rp, (size_t)n_pre + 1, "row starts"));
        TRY(dalloc(net, &col, padded, "post indices"));
        TRY(dalloc(net, &w, padded, "weights"));
        CK(cudaMemsetAsync(col, 0, padded * sizeof(int32_t), s), "clear");
        CK(cudaMemsetAsync(w, 0, padded * sizeof(float), s), "clear");
        CK(cudaMemcpyAsync(rp, P.d.row_ptr, sizeof(int64_t) * ((size_t)n_pre + 1), kind, s), "copy row starts");
        if (P.nnz > 0) {
            CK(cudaMemcpyAsync(col, P.d.col, sizeof(int32_t) * P.nnz, kind, s), "copy post indices");
            CK(cudaMemcpyAsync(w, P.d.w, sizeof(float) * P.nnz, kind, s), "copy weights");
        }
        CK(launch_validate_csr(rp, col, n_pre, n_post, P.nnz, net->error, s), "validate rows");
        P.row_ptr = rp;
        P.col = col;
        P.w = w;
    }
    TRY(sticky(net, s));       // connectivity is checked before any kernel indexes with it
    for (int q = 0; q < n_projs; ++q) {
        ProjHost& P = net->projs[q];
        if (P.d.input_dense) continue;
        const int32_t n_pre = pops[P.d.pre].n, n_post = pops[P.d.post].n;
        CK(launch_max_row(P.row_ptr, n_pre, d_max + q, s), "row maximum");
        if (P.d.layout == SNN_LAYOUT_DENSE) {
            float* W = nullptr;
            const size_t cnt = (size_t)n_pre * n_post;
            TRY(dalloc(net, &W, cnt + 4, "dense weights"));
            CK(cudaMemsetAsync(W, 0, (cnt + 4) * sizeof(float), s), "clear");
            CK(launch_densify(P.row_ptr, P.col, P.w, n_pre, n_post, W, s), "densify");
            P.w = W;
            P.nnz = (int64_t)cnt;
        }
    }
    if (n_projs > 0) {
        std::vector<int32_t> mx((size_t)n_projs);
        CK(cudaMemcpyAsync(mx.data(), d_max, sizeof(int32_t) * n_projs, cudaMemcpyDeviceToHost, s), "read maxima");
        CK(cudaStreamSynchronize(s), "synchronize");
        for (int q = 0; q < n_projs; ++q) net->projs[q].max_row = mx[q];
    }
    {   // projections grouped by pre population, for the persistent engine's pushes
        std::vector<int32_t> begin((size_t)n_pops + 1, 0), list;
        for (int k = 0; k < n_pops; ++k) {
            begin[k] = (int32_t)list.size();
            for (int q = 0; q < n_projs; ++q)
                if (net->projs[q].d.pre == k) list.push_back(q);
        }
        begin[n_pops] = (int32_t)list.size();
        if (list.empty()) list.push_back(0);
        CK(cudaMemcpyAsync(net->out_begin, begin.data(), begin.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s),
           "upload outgoing offsets");
        CK(cudaMemcpyAsync(net->out_list, list.data(), list.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s),
           "upload outgoing projections");
        CK(cudaStreamSynchronize(s), "synchronize");
    }
    CK(persistent_capacity(net->sm_count, &net->persist_grid), "persistent occupancy");
    {
        int per = 0;
        const int cl = cluster_plan(net->num_tiles * kTile, n_pops, n_projs, &per);
        // compressed rows, in projection order, whose segments fit the shared cache
        int seg_rows = 0;
        for (int q = 0; q < n_projs; ++q) {
            if (net->projs[q].d.layout != SNN_LAYOUT_CSR) continue;
            const int n_pre = pops[net->projs[q].d.pre].n;
            if (seg_rows + n_pre > kClusterSegCacheRows) break;
            seg_rows += n_pre;
        }
        bool ok = false;
        if (cl && !graded_requested(projs, n_projs))
            CK(cluster_supported(cl, per, net->num_tiles, seg_rows, &ok), "cluster occupancy");
        net->cluster_size = ok ? cl : 0;
        net->cluster_per_cta = ok ? per : 0;
        net->cluster_seg_rows = ok ? seg_rows : 0;
        for (int q = 0; ok && q < n_projs; ++q) {   // each row's segment in each CTA's slice
            ProjHost& P = net->projs[q];
            if (P.d.layout != SNN_LAYOUT_CSR) continue;
            const int32_t n_pre = pops[P.d.pre].n, n_post = pops[P.d.post].n;
            TRY(dalloc(net, &P.csplit, (size_t)n_pre * (cl + 1) + 1, "cluster row segments"));
            CK(launch_cluster_splits(P.row_ptr, P.col, n_pre, net->pops[P.d.post].offset, n_post, cl, per, P.csplit,
                                     s), "cluster row segments");
        }
    }
    TRY(setup_tiled(net, s));
    if (graded_requested(projs, n_projs)) TRY(graded_setup(net, s));
    // save the creation state for snn_reset
    CK(cudaMemcpyAsync(net->init_state, net->V, 7 * NT * sizeof(float), cudaMemcpyDeviceToDevice, s),
       "save initial state");
    CK(cudaStreamSynchronize(s), "synchronize");
    guard.net = nullptr;
    *out = net;
    return SNN_OK;
}

}  // namespace

namespace snn {

// Marks channel 1 and the drive current of population `pop` (all
// populations for pop < 0) as possibly nonzero, so the step kernels read and
// write them from then on.
cudaError_t mark_state_live(snn_net* net, int32_t pop, bool g1, bool iext, cudaStream_t s) {
    static const int32_t one = 1;
    const int32_t lo = pop < 0 ? 0 : pop, hi = pop < 0 ? (int32_t)net->pops.size() : pop + 1;
    for (int32_t k = lo; k < hi; ++k) {
        DevPop* d = net->d_pops + k;
        cudaError_t e = cudaSuccess;
        if (g1) e = cudaMemcpyAsync(&d->g1_live, &one, sizeof(int32_t), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && iext) e = cudaMemcpyAsync(&d->iext_live, &one, sizeof(int32_t), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace snn

// ===========================================================================
// C-ABI
// ===========================================================================
extern "C" {

const char* snn_last_error(void) { return g_err.c_str(); }

snn_status snn_create_network(const snn_pop_desc* pops, int32_t n_pops, const snn_proj_desc* projs,
                              int32_t n_projs, double dt, int32_t n_substeps, uint64_t seed,
                              uint32_t rng_instance, const snn_allocator* alloc, void* stream,
                              snn_net** out) {
    try {
        if (rng_instance >= (1u << 24)) return fail(SNN_ERR_INVALID_ARG, "rng_instance must be < 2^24");
        if (n_pops > 256) return fail(SNN_ERR_INVALID_ARG, "a single instance has at most 256 populations");
        std::vector<uint32_t> tags((size_t)std::max(n_pops, 0));
        for (int k = 0; k < n_pops; ++k) tags[k] = (rng_instance << 8) | (uint32_t)k;
        return create_impl(pops, n_pops, projs, n_projs, dt, n_substeps, seed, tags, alloc, (cudaStream_t)stream,
                           out);
    } catch (const std::bad_alloc&) {
        return fail(SNN_ERR_OOM, "host allocation failed");
    } catch (...) {
        return fail(SNN_ERR_INVALID_ARG, "unexpected host exception");
    }
}

snn_status snn_create_batch(const snn_net_desc* nets, int32_t n_instances, double dt, int32_t n_substeps,
                            uint64_t seed, const snn_allocator* alloc, void* stream, snn_net** out) {
    try {
        if (!nets || n_instances < 1) return fail(SNN_ERR_INVALID_ARG, "need at least one instance");
        std::vector<snn_pop_desc> pops;
        std::vector<snn_proj_desc> projs;
        std::vector<uint32_t> tags;
        for (int b = 0; b < n_instances; ++b) {
            const snn_net_desc& d = nets[b];
            if (d.n_pops < 1 || d.n_pops > 256 || !d.pops || d.n_projs < 0 || (d.n_projs > 0 && !d.projs))
                return fail(SNN_ERR_INVALID_ARG, "instance " + std::to_string(b) + ": bad populations or projections");
            if (d.rng_instance >= (1u << 24)) return fail(SNN_ERR_INVALID_ARG, "rng_instance must be < 2^24");
            const int32_t base = (int32_t)pops.size();
            if (base + d.n_pops > kMaxPops || (int64_t)projs.size() + d.n_projs > kMaxProjs)
                return fail(SNN_ERR_INVALID_ARG, "at most 4096 populations and 4096 projections in a batch");
            for (int k = 0; k < d.n_pops; ++k) {
                pops.push_back(d.pops[k]);
                tags.push_back((d.rng_instance << 8) | (uint32_t)k);
            }
            for (int q = 0; q < d.n_projs; ++q) {
                snn_proj_desc p = d.projs[q];
                if (p.pre < 0 || p.pre >= d.n_pops || p.post < 0 || p.post >= d.n_pops)
                    return fail(SNN_ERR_INVALID_ARG, "instance " + std::to_string(b) + ": projection outside the instance");
                p.pre += base;
                p.post += base;
                projs.push_back(p);
            }
        }
        return create_impl(pops.data(), (int32_t)pops.size(), projs.empty() ? nullptr : projs.data(),
                           (int32_t)projs.size(), dt, n_substeps, seed, tags, alloc, (cudaStream_t)stream, out);
    } catch (const std::bad_alloc&) {
        return fail(SNN_ERR_OOM, "host allocation failed");
    } catch (...) {
        return fail(SNN_ERR_INVALID_ARG, "unexpected host exception");
    }
}

snn_status snn_destroy(snn_net* net) {
    if (!net) return SNN_OK;
    cudaDeviceSynchronize();
    for (SharedDense& d : net->shared) snn_dense_batch_destroy(d.h);
    net->shared.clear();
    release(net);
    delete net;
    return SNN_OK;
}

snn_status snn_step(snn_net* net, int64_t n_steps, void* stream) {
    if (!net || n_steps < 0) return fail(SNN_ERR_INVALID_ARG, "bad network or step count");
    cudaStream_t s = (cudaStream_t)stream;
    try {
        if (net->graded) return graded_step(net, n_steps, s);
        if (use_cluster(net)) {
            for (int64_t left = n_steps; left > 0;) {
                const int32_t k = (int32_t)std::min<int64_t>(left, net->persist_steps);
                CK(launch_cluster(persist_args(net, k), net->cluster_size, net->cluster_per_cta,
                                  (int)net->projs.size(), net->cluster_seg_rows, s), "cluster steps");
                left -= k;
            }
            return SNN_OK;
        }
        if (use_persistent(net)) {
            CK(enqueue_persistent(net, n_steps, s), "persistent steps");
            return SNN_OK;
        }
        int64_t left = n_steps;
        if (net->graph_steps > 0 && left >= net->graph_steps) {
            TRY(ensure_graph(net));
            while (left >= net->graph_steps) {
                CK(cudaGraphLaunch(net->graph, s), "launch graph");
                left -= net->graph_steps;
            }
        }
        for (; left > 0; --left) CK(enqueue_step(net, s), "launch step");
    } catch (...) {
        return fail(SNN_ERR_INVALID_ARG, "unexpected host exception");
    }
    return SNN_OK;
}

snn_status snn_sync(snn_net* net, void* stream) {
    if (!net) return fail(SNN_ERR_INVALID_ARG, "net is NULL");
    return sticky(net, (cudaStream_t)stream);
}

snn_status snn_read_state(snn_net* net, int32_t pop, int32_t field, void* dst, size_t bytes,
                          int32_t dst_is_device, void* stream) {
    if (!net || !dst || pop < 0 || pop >= (int32_t)net->pops.size())
        return fail(SNN_ERR_INVALID_ARG, "bad network, population or destination");
    cudaStream_t s = (cudaStream_t)stream;
    const PopHost& P = net->pops[pop];
    const cudaMemcpyKind kind = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    TRY(sticky(net, s));
    if (field >= SNN_FIELD_V && field <= SNN_FIELD_ISYN) {
        const size_t need = sizeof(float) * (size_t)P.d.n;
        if (bytes < need) return fail(SNN_ERR_SIZE, "destination smaller than n floats");
        if (P.d.n) CK(cudaMemcpyAsync(dst, field_base(net, field) + P.offset, need, kind, s), "copy field");
    } else if (field == SNN_FIELD_NSPK || field == SNN_FIELD_SPIKES) {
        // the list of the last completed step: parity slot of epoch ticket / num_tiles - 1
        unsigned long long tk = 0;
        int32_t cnt[2] = {0, 0};
        CK(cudaMemcpyAsync(&tk, net->ticket, sizeof(tk), cudaMemcpyDeviceToHost, s), "read ticket");
        CK(cudaMemcpyAsync(cnt, net->nspk + 2 * pop, sizeof(cnt), cudaMemcpyDeviceToHost, s), "read counts");
        CK(cudaStreamSynchronize(s), "synchronize");
        const unsigned long long done = net->num_tiles ? tk / (unsigned long long)net->num_tiles : 0;
        const int32_t ns = done ? cnt[(done - 1) & 1] : 0;
        if (field == SNN_FIELD_NSPK) {
            if (bytes < sizeof(int32_t)) return fail(SNN_ERR_SIZE, "destination smaller than 4 bytes");
            CK(cudaMemcpyAsync(dst, &ns, sizeof(int32_t), dst_is_device ? cudaMemcpyHostToDevice
                                                                           : cudaMemcpyHostToHost, s), "copy count");
        } else {
            if (bytes < sizeof(int32_t) * (size_t)ns) return fail(SNN_ERR_SIZE, "destination smaller than the spike list");
            std::vector<int32_t> list((size_t)ns);
            if (ns) {
                CK(cudaMemcpyAsync(list.data(), net->spk + P.offset, sizeof(int32_t) * ns, cudaMemcpyDeviceToHost, s),
                   "copy spikes");
                CK(cudaStreamSynchronize(s), "synchronize");
                std::sort(list.begin(), list.end());      // ascending neuron index
                CK(cudaMemcpyAsync(dst, list.data(), sizeof(int32_t) * ns,
                                   dst_is_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, s), "copy spikes");
            }
        }
    } else if (field == SNN_FIELD_NEURON_SPIKES) {
        const size_t need = sizeof(int32_t) * (size_t)P.d.n;
        if (bytes < need) return fail(SNN_ERR_SIZE, "destination smaller than n int32");
        if (P.d.n) CK(cudaMemcpyAsync(dst, net->nrn_count + P.offset, need, kind, s), "copy counts");
    } else if (field == SNN_FIELD_SPIKE_COUNT || field == SNN_FIELD_NAN_COUNT) {
        if (bytes < sizeof(int64_t)) return fail(SNN_ERR_SIZE, "destination smaller than 8 bytes");
        const int o = field == SNN_FIELD_SPIKE_COUNT ? 0 : 1;
        CK(cudaMemcpyAsync(dst, net->counters + 2 * pop + o, sizeof(int64_t), kind, s), "copy counter");
    } else {
        return fail(SNN_ERR_INVALID_ARG, "unknown field");
    }
    CK(cudaStreamSynchronize(s), "synchronize");
    return SNN_OK;
}

snn_status snn_write_state(snn_net* net, int32_t pop, int32_t field, const void* src, size_t bytes,
                           int32_t src_is_device, void* stream) {
    if (!net || !src || pop < 0 || pop >= (int32_t)net->pops.size())
        return fail(SNN_ERR_INVALID_ARG, "bad network, population or source");
    if (field < SNN_FIELD_V || field > SNN_FIELD_IEXT) return fail(SNN_ERR_INVALID_ARG, "field is not writable");
    const PopHost& P = net->pops[pop];
    const size_t need = sizeof(float) * (size_t)P.d.n;
    if (bytes != need) return fail(SNN_ERR_SIZE, "source must hold exactly n floats");
    cudaStream_t s = (cudaStream_t)stream;
    if (P.d.n)
        CK(cudaMemcpyAsync(field_base(net, field) + P.offset, src, need,
                           src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s),
           "write field");
    if (field == SNN_FIELD_G1 || field == SNN_FIELD_IEXT)
        CK(mark_state_live(net, pop, field == SNN_FIELD_G1, field == SNN_FIELD_IEXT, s), "mark field live");
    CK(cudaStreamSynchronize(s), "synchronize");
    return SNN_OK;
}

snn_status snn_reset(snn_net* net, void* stream) {
    if (!net) return fail(SNN_ERR_INVALID_ARG, "net is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t NT = std::max<size_t>(1, (size_t)net->n_total);
    CK(cudaMemcpyAsync(net->V, net->init_state, 7 * NT * sizeof(float), cudaMemcpyDeviceToDevice, s), "restore");
    CK(cudaMemsetAsync(net->isyn, 0, NT * sizeof(float), s), "clear");
    CK(cudaMemsetAsync(net->nspk, 0, sizeof(int32_t) * 2 * net->pops.size(), s), "clear");
    CK(cudaMemsetAsync(net->counters, 0, sizeof(unsigned long long) * 2 * net->pops.size(), s), "clear");
    CK(cudaMemsetAsync(net->nrn_count, 0, NT * sizeof(int32_t), s), "clear");
    CK(cudaMemsetAsync(net->acc, 0, 4 * NT * sizeof(float), s), "clear");
    CK(cudaMemsetAsync(net->bar, 0, sizeof(GridBarrier), s), "clear");
    CK(cudaMemsetAsync(net->error, 0, sizeof(uint32_t), s), "clear");
    CK(launch_set_epoch_base(net->ticket, net->num_tiles, s), "reset step counter");
    if (net->graded) return graded_reset(net, s);
    return SNN_OK;
}

snn_status snn_get_option(const snn_net* net, int32_t option, int64_t* value) {
    if (!net || !value) return fail(SNN_ERR_INVALID_ARG, "net or value is NULL");
    switch (option) {
    case SNN_OPT_RECORD_ISYN: *value = net->record_isyn ? 1 : 0; break;
    case SNN_OPT_GRAPH_STEPS: *value = net->graph_steps; break;
    case SNN_OPT_PROP_BLOCKS: *value = net->prop_blocks; break;
    case SNN_OPT_CHUNK: *value = net->chunk; break;
    case SNN_OPT_SPIN_LIMIT: *value = net->spin_limit; break;
    case SNN_OPT_ENGINE: *value = net->engine; break;
    case SNN_OPT_PERSIST_STEPS: *value = net->persist_steps; break;
    case SNN_OPT_TILED: *value = net->tiled; break;
    case SNN_OPT_TEST_BARRIER_EXTRA: *value = net->barrier_extra; break;
    case SNN_OPT_CLUSTER_CTAS: *value = net->cluster_size; break;
    case SNN_OPT_DENSE_GRAD: *value = net->dense_grad; break;
    case SNN_OPT_SHARED_DENSE: *value = net->shared_engine; break;
    case SNN_OPT_GRADED_STORE: *value = net->graded_store; break;
    default: return fail(SNN_ERR_INVALID_ARG, "unknown option");
    }
    return SNN_OK;
}

snn_status snn_set_option(snn_net* net, int32_t option, int64_t value) {
    if (!net) return fail(SNN_ERR_INVALID_ARG, "net is NULL");
    switch (option) {
    case SNN_OPT_RECORD_ISYN: net->record_isyn = value != 0; break;
    case SNN_OPT_GRAPH_STEPS:
        if (value < 0 || value > 100000) return fail(SNN_ERR_INVALID_ARG, "graph steps in 0..100000");
        net->graph_steps = value;
        break;
    case SNN_OPT_PROP_BLOCKS:
        if (value < 0 || value > 65535) return fail(SNN_ERR_INVALID_ARG, "blocks in 0..65535");
        net->prop_blocks = (int32_t)value;
        break;
    case SNN_OPT_CHUNK:
        if (value < 128 || value > (1 << 24) || value % 128) return fail(SNN_ERR_INVALID_ARG, "chunk: multiple of 128");
        net->chunk = (int32_t)value;
        TRY(upload_projs(net));
        break;
    case SNN_OPT_SPIN_LIMIT:
        if (value < 1 || value > (int64_t)1 << 31) return fail(SNN_ERR_INVALID_ARG, "spin limit in 1..2^31");
        net->spin_limit = (uint32_t)value;
        break;
    case SNN_OPT_ENGINE:
        if (value < 0 || value > 3) return fail(SNN_ERR_INVALID_ARG, "engine: 0 plain, 1 persistent, 2 choose, 3 cluster");
        if (value == 1 && net->persist_grid <= 0) return fail(SNN_ERR_STATE, "persistent kernel cannot be resident");
        if (value == 3 && net->cluster_size == 0) return fail(SNN_ERR_STATE, "network does not fit one cluster");
        net->engine = (int32_t)value;
        break;
    case SNN_OPT_TEST_BARRIER_EXTRA:
        if (value < 0 || value > 1) return fail(SNN_ERR_INVALID_ARG, "test barrier hook: 0 or 1");
        net->barrier_extra = (int32_t)value;
        break;
    case SNN_OPT_TILED:
        if (value < 0 || value > 3) return fail(SNN_ERR_INVALID_ARG, "tiled: 0 off, 1 bulk copies, 2 choose, 3 segments");
        net->tiled = (int32_t)value;
        TRY(setup_tiled(net, nullptr));
        break;
    case SNN_OPT_PERSIST_STEPS:
        if (value < 1 || value > (1 << 24)) return fail(SNN_ERR_INVALID_ARG, "persistent steps in 1..2^24");
        net->persist_steps = (int32_t)value;
        break;
    case SNN_OPT_DENSE_GRAD:
        if (value < 0 || value > 1) return fail(SNN_ERR_INVALID_ARG, "dense gradient: 0 CUDA cores, 1 tensor cores");
        net->dense_grad = (int32_t)value;
        break;
    case SNN_OPT_GRADED_STORE:
        if (value < 0 || value > 1) return fail(SNN_ERR_INVALID_ARG, "graded store: 0 recompute, 1 store when it fits");
        net->graded_store = (int32_t)value;
        break;
    case SNN_OPT_SHARED_DENSE:
        if (value < 0 || value > 2) return fail(SNN_ERR_INVALID_ARG, "shared dense: 0 CUDA cores, 1 tensor cores, 2 by density");
        net->shared_engine = (int32_t)value;
        drop_graph(net);
        break;
    default: return fail(SNN_ERR_INVALID_ARG, "unknown option");
    }
    drop_graph(net);
    return SNN_OK;
}

snn_status snn_get_engine(snn_net* net, int32_t* engine) {
    if (!net || !engine) return fail(SNN_ERR_INVALID_ARG, "bad argument");
    *engine = net->graded ? 0 : use_cluster(net) ? 3 : use_persistent(net) ? 1 : 0;
    return SNN_OK;
}

snn_status snn_get_step(snn_net* net, int64_t* step, void* stream) {
    if (!net || !step) return fail(SNN_ERR_INVALID_ARG, "bad argument");
    unsigned long long t[2];
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(t, net->ticket, sizeof(t), cudaMemcpyDeviceToHost, s), "read ticket");
    CK(cudaStreamSynchronize(s), "synchronize");
    *step = net->graded ? net->g_t : net->num_tiles ? (int64_t)(t[0] / (unsigned long long)net->num_tiles - t[1]) : 0;
    return SNN_OK;
}

snn_status snn_synaptic_events(snn_net* net, int64_t* events, void* stream) {
    if (!net || !events) return fail(SNN_ERR_INVALID_ARG, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long v = 0;
    CK(launch_count_events(net->d_projs, (int)net->projs.size(), net->d_events, s), "count events");
    CK(cudaMemcpyAsync(&v, net->d_events, sizeof(v), cudaMemcpyDeviceToHost, s), "read events");
    std::vector<unsigned long long> cnt;
    if (!net->shared.empty()) {                    // shared dense rows: spikes of the pre populations x n_post
        cnt.resize(2 * net->pops.size());
        CK(cudaMemcpyAsync(cnt.data(), net->counters, sizeof(unsigned long long) * cnt.size(), cudaMemcpyDeviceToHost, s),
           "read counters");
    }
    CK(cudaStreamSynchronize(s), "synchronize");
    for (const SharedDense& d : net->shared)
        for (int32_t p : d.pre_pops) v += cnt[2 * (size_t)p] * (unsigned long long)d.n_post;
    *events = (int64_t)v;
    return SNN_OK;
}

snn_status snn_launch_phase(snn_net* net, int32_t phase, void* stream) {
    if (!net || phase < 0 || phase > 4) return fail(SNN_ERR_INVALID_ARG, "bad network or phase");
    cudaStream_t s = (cudaStream_t)stream;
    if (phase == 4) {
        if (net->cluster_size == 0) return fail(SNN_ERR_STATE, "network does not fit one cluster");
        CK(launch_cluster(persist_args(net, net->persist_steps), net->cluster_size, net->cluster_per_cta,
                          (int)net->projs.size(), net->cluster_seg_rows, s),
           "cluster phase");
    } else if (phase == 3) {
        if (!net->dbg_staged) return fail(SNN_ERR_STATE, "no spike list staged by snn_debug_propagate");
        const ProjHost* h = &net->projs[net->dbg_proj];
        CK(launch_projections(net, net->d_dbg_proj, &h, 1, s), "staged propagation");
    } else if (phase == 2) {
        if (net->persist_grid <= 0) return fail(SNN_ERR_STATE, "persistent kernel cannot be resident");
        CK(launch_persistent(persist_args(net, net->persist_steps), net->persist_grid, s), "persistent phase");
    } else if (phase == 0) {
        CK(launch_neuron_step(neuron_args(net), s), "neuron phase");
    } else {
        CK(launch_all_projections(net, s), "propagation phase");
    }
    return SNN_OK;
}

snn_status snn_proj_scale(snn_net* net, int32_t proj, float* scale) {
    if (!net || !scale || proj < 0 || proj >= (int32_t)net->projs.size()) return fail(SNN_ERR_INVALID_ARG, "bad argument");
    *scale = net->projs[proj].scale;
    return SNN_OK;
}

snn_status snn_proj_mode(snn_net* net, int32_t proj, int32_t* mode) {
    if (!net || !mode || proj < 0 || proj >= (int32_t)net->projs.size()) return fail(SNN_ERR_INVALID_ARG, "bad argument");
    *mode = net->projs[proj].mode;
    return SNN_OK;
}

snn_status snn_proj_nnz(snn_net* net, int32_t proj, int64_t* nnz) {
    if (!net || !nnz || proj < 0 || proj >= (int32_t)net->projs.size()) return fail(SNN_ERR_INVALID_ARG, "bad argument");
    *nnz = net->projs[proj].nnz;
    return SNN_OK;
}

static snn_status stage_spikes(snn_net* net, int32_t proj, const int32_t* spk, int32_t n, int32_t on_device,
                               cudaStream_t s) {
    const int32_t n_pre = net->pops[net->projs[proj].d.pre].d.n;
    if (n < 0 || n > n_pre) return fail(SNN_ERR_INVALID_ARG, "spike count out of range");
    if (n > 0 && !spk) return fail(SNN_ERR_INVALID_ARG, "spike list is NULL");
    std::vector<int32_t> h((size_t)n);
    if (n) {
        if (on_device) {
            CK(cudaMemcpyAsync(h.data(), spk, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s), "read spikes");
            CK(cudaStreamSynchronize(s), "synchronize");
        } else {
            std::memcpy(h.data(), spk, sizeof(int32_t) * n);
        }
    }
    for (int32_t k = 0; k < n; ++k)
        if (h[k] < 0 || h[k] >= n_pre || (k && h[k] <= h[k - 1]))
            return fail(SNN_ERR_INVALID_ARG, "spike list must be ascending indices of the pre population");
    if (net->dbg_cap < n + 2) {
        int32_t* p = nullptr;
        TRY(dalloc(net, &p, (size_t)n + 2, "debug spikes"));
        net->d_dbg_spk = p;
        net->dbg_cap = n + 2;
    }
    h.push_back(n);   // the count, in both parity slots, after the list
    h.push_back(n);
    CK(cudaMemcpyAsync(net->d_dbg_spk, h.data(), sizeof(int32_t) * (n + 2), cudaMemcpyHostToDevice, s), "stage");
    CK(cudaStreamSynchronize(s), "synchronize");
    return SNN_OK;
}

snn_status snn_debug_propagate(snn_net* net, int32_t proj, const int32_t* spk, int32_t n, int32_t spk_on_device,
                               void* stream) {
    if (!net || proj < 0 || proj >= (int32_t)net->projs.size()) return fail(SNN_ERR_INVALID_ARG, "bad projection");
    cudaStream_t s = (cudaStream_t)stream;
    try {
        TRY(stage_spikes(net, proj, spk, n, spk_on_device, s));
        DevProj d;
        CK(cudaMemcpyAsync(&d, net->d_projs + proj, sizeof(d), cudaMemcpyDeviceToHost, s), "read descriptor");
        CK(cudaStreamSynchronize(s), "synchronize");
        d.spk = net->d_dbg_spk;
        d.nspk = net->d_dbg_spk + n;
        CK(cudaMemcpyAsync(net->d_dbg_proj, &d, sizeof(d), cudaMemcpyHostToDevice, s), "write descriptor");
        net->dbg_staged = true;
        net->dbg_proj = proj;
        const ProjHost* h = &net->projs[proj];
        CK(launch_projections(net, net->d_dbg_proj, &h, 1, s), "propagate");
        return sticky(net, s);
    } catch (...) {
        return fail(SNN_ERR_OOM, "host allocation failed");
    }
}

snn_status snn_event_list(snn_net* net, int32_t proj, const int32_t* spk, int32_t n, int32_t spk_on_device,
                          int32_t* post_out, float* w_out, int64_t capacity, int64_t* n_events, void* stream) {
    if (!net || proj < 0 || proj >= (int32_t)net->projs.size() || !n_events)
        return fail(SNN_ERR_INVALID_ARG, "bad argument");
    const ProjHost& P = net->projs[proj];
    if (P.d.layout != SNN_LAYOUT_CSR) return fail(SNN_ERR_INVALID_ARG, "event lists need compressed rows");
    cudaStream_t s = (cudaStream_t)stream;
    try {
        TRY(stage_spikes(net, proj, spk, n, spk_on_device, s));
        int64_t* lens = nullptr;
        int64_t* offs = nullptr;
        int64_t* scratch = nullptr;
        void* a = net->mem.get(sizeof(int64_t) * ((size_t)n + 1));
        void* b = net->mem.get(sizeof(int64_t) * ((size_t)n + 1));
        void* c = net->mem.get(sizeof(int64_t) * scan_scratch_elems(n));
        auto cleanup = [&]() { net->mem.put(a); net->mem.put(b); net->mem.put(c); };
        if (!a || !b || !c) {
            cleanup();
            return fail(SNN_ERR_OOM, "event list scratch");
        }
        lens = (int64_t*)a; offs = (int64_t*)b; scratch = (int64_t*)c;
        cudaError_t e = launch_row_lengths(P.row_ptr, net->d_dbg_spk, n, lens, s);
        if (e == cudaSuccess) e = launch_scan_i64(lens, offs, n, scratch, s);
        int64_t total = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&total, offs + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            cleanup();
            return cuda_fail(e, "event offsets");
        }
        *n_events = total;
        if (total > capacity || (total > 0 && (!post_out || !w_out))) {
            cleanup();
            return fail(SNN_ERR_SIZE, "event list larger than capacity");
        }
        e = launch_event_list(P.row_ptr, P.col, P.w, net->d_dbg_spk, n, offs, post_out, w_out, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cleanup();
        if (e != cudaSuccess) return cuda_fail(e, "event list");
        return SNN_OK;
    } catch (...) {
        return fail(SNN_ERR_OOM, "host allocation failed");
    }
}

snn_status snn_csr_bernoulli_rows(uint64_t seed, uint32_t tag, int64_t n_pre, int64_t n_post, double p,
                                  int64_t* row_ptr, int64_t* nnz, const snn_allocator* alloc, void* stream) {
    if (n_pre < 0 || n_post < 0 || n_pre >= (int64_t(1) << 31) || n_post >= (int64_t(1) << 31) || !(p >= 0.0) ||
        p > 1.0 || !row_ptr || !nnz)
        return fail(SNN_ERR_INVALID_ARG, "bad sizes, probability or pointers");
    cudaStream_t s = (cudaStream_t)stream;
    Alloc mem;
    if (alloc) {
        if (!alloc->alloc || !alloc->free) return fail(SNN_ERR_INVALID_ARG, "allocator without alloc/free");
        mem.a = *alloc;
        mem.have = true;
    }
    mem.stream = s;
    int64_t* counts = (int64_t*)mem.get(sizeof(int64_t) * std::max<int64_t>(1, n_pre));
    int64_t* scratch = (int64_t*)mem.get(sizeof(int64_t) * scan_scratch_elems(n_pre));
    if (!counts || !scratch) {
        mem.put(counts);
        mem.put(scratch);
        return fail(SNN_ERR_OOM, "scratch allocation failed");
    }
    const unsigned long long thr = bernoulli_threshold(p);
    cudaError_t e = launch_csr_count(seed, tag, n_pre, n_post, thr, counts, s);
    if (e == cudaSuccess) e = launch_scan_i64(counts, row_ptr, n_pre, scratch, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(nnz, row_ptr + n_pre, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    mem.put(counts);
    mem.put(scratch);
    if (e != cudaSuccess) return cuda_fail(e, "draw rows");
    return SNN_OK;
}

snn_status snn_csr_bernoulli_fill(uint64_t seed, uint32_t tag, int64_t n_pre, int64_t n_post, double p,
                                  const int64_t* row_ptr, int32_t* col, void* stream) {
    if (n_pre < 0 || n_post < 0 || n_pre >= (int64_t(1) << 31) || n_post >= (int64_t(1) << 31) || !(p >= 0.0) ||
        p > 1.0 || !row_ptr || (!col && n_pre > 0 && n_post > 0 && p > 0.0))
        return fail(SNN_ERR_INVALID_ARG, "bad sizes, probability or pointers");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = launch_csr_fill(seed, tag, n_pre, n_post, bernoulli_threshold(p), row_ptr, col, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "fill rows");
    return SNN_OK;
}

snn_status snn_add_shared_dense(snn_net* net, int32_t first_pre, int32_t first_post, int32_t pops_per_instance,
                                int32_t n_instances, const float* w, int32_t w_on_device, int32_t channel, double k1,
                                double k2, double k3, double density, double n_conn, const double* user_scale,
                                void* stream) {
    if (!net || !w || !user_scale || n_instances < 1 || pops_per_instance < 1 || (channel != 0 && channel != 1))
        return fail(SNN_ERR_INVALID_ARG, "shared dense: bad network, weights, scales, instance layout or channel");
    if (net->graded) return fail(SNN_ERR_STATE, "shared dense: not for graded networks");
    const int32_t np = (int32_t)net->pops.size(), B = n_instances;
    if (first_pre < 0 || first_post < 0 || first_pre >= pops_per_instance || first_post >= pops_per_instance ||
        (int64_t)(B - 1) * pops_per_instance + std::max(first_pre, first_post) >= np)
        return fail(SNN_ERR_INVALID_ARG, "shared dense: populations outside the batch");
    const int32_t n_pre = net->pops[first_pre].d.n, n_post = net->pops[first_post].d.n;
    const int64_t off0 = net->pops[first_post].offset;
    const int64_t ldg = B > 1 ? (int64_t)net->pops[first_post + pops_per_instance].offset - off0 : (int64_t)n_post;
    std::vector<int32_t> pre_pop((size_t)B), pre_off((size_t)B);
    std::vector<float> scale((size_t)B);
    const double nc = n_conn > 0.0 ? n_conn : density * (double)n_pre;
    if (!(k2 + nc > 0.0) || !std::isfinite(k2 + nc)) return fail(SNN_ERR_GSCALE, "shared dense: nConn + k2 <= 0");
    for (int32_t b = 0; b < B; ++b) {
        const int32_t pp = first_pre + b * pops_per_instance, qp = first_post + b * pops_per_instance;
        if (net->pops[pp].d.n != n_pre || net->pops[qp].d.n != n_post)
            return fail(SNN_ERR_INVALID_ARG, "shared dense: instance " + std::to_string(b) + " has other population sizes");
        if (net->pops[qp].d.kind == SNN_POP_SOURCE)
            return fail(SNN_ERR_INVALID_ARG, "shared dense: the post population must not be a source");
        if ((int64_t)net->pops[qp].offset != off0 + b * ldg)
            return fail(SNN_ERR_INVALID_ARG, "shared dense: post populations are not evenly spaced (instances differ)");
        pre_pop[b] = pp;
        pre_off[b] = net->pops[pp].offset;
        const double sv = (k1 / (k2 + nc) + k3) * user_scale[b];
        if (!std::isfinite(sv)) return fail(SNN_ERR_GSCALE, "shared dense: non-finite scale");
        scale[b] = (float)sv;
    }
    cudaStream_t s = (cudaStream_t)stream;
    try {
        SharedDense d;
        d.B = B;
        d.n_pre = n_pre;
        d.n_post = n_post;
        d.channel = channel;
        d.ldg = ldg;
        d.G = (channel == 0 ? net->g0 : net->g1) + off0;
        d.pre_pops = pre_pop;
        snn_status st = snn_dense_batch_create(w, n_pre, n_post, w_on_device, net->mem.have ? &net->mem.a : nullptr,
                                               stream, &d.h);
        if (st != SNN_OK) return st;
        struct Undo {
            SharedDense* d;
            ~Undo() { if (d) snn_dense_batch_destroy(d->h); }
        } undo{&d};
        TRY(dense_batch_reserve(d.h, B, s));
        TRY(dalloc(net, &d.pre_pop, (size_t)B, "shared pre populations"));
        TRY(dalloc(net, &d.pre_off, (size_t)B, "shared pre offsets"));
        TRY(dalloc(net, &d.spk_off, (size_t)B + 1, "shared spike offsets"));
        TRY(dalloc(net, &d.spk, (size_t)B * n_pre, "shared spike lists"));
        TRY(dalloc(net, &d.scale, (size_t)B, "shared scales"));
        CK(cudaMemcpyAsync(d.pre_pop, pre_pop.data(), sizeof(int32_t) * B, cudaMemcpyHostToDevice, s), "upload");
        CK(cudaMemcpyAsync(d.pre_off, pre_off.data(), sizeof(int32_t) * B, cudaMemcpyHostToDevice, s), "upload");
        CK(cudaMemcpyAsync(d.scale, scale.data(), sizeof(float) * B, cudaMemcpyHostToDevice, s), "upload");
        if (channel == 1)
            for (int32_t b = 0; b < B; ++b) CK(mark_state_live(net, first_post + b * pops_per_instance, true, false, s),
                                               "channel 1 live");
        CK(cudaStreamSynchronize(s), "synchronize");
        undo.d = nullptr;
        net->shared.push_back(d);
        drop_graph(net);
        if (net->engine == 1 || net->engine == 3) net->engine = 2;
        return SNN_OK;
    } catch (const std::bad_alloc&) {
        return fail(SNN_ERR_OOM, "host allocation failed");
    }
}

}  // extern "C"
