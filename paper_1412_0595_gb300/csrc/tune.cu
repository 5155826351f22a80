// State snapshots (checkpoint / resume) and the autotuner.
//
// A snapshot holds everything a step reads or writes: the structure-of-arrays
// state, spike lists and their double-buffered lengths, per-neuron and
// per-population counters, the persistent engine's event accumulators and
// barrier counter, and the step ticket (hence the random-number counters).
// Loading it and stepping reproduces the uninterrupted run up to the order of
// floating-point atomic adds.
//
// The autotuner times candidate launch configurations -- engine (plain /
// persistent / cluster), propagation CTAs, compressed-row chunk, post-tiled rows -- on
// short trial runs from a snapshot of the live network, keeps the fastest,
// and restores the snapshot, so tuning never changes the trajectory.  Results
// are cached per device and network shape for the life of the process.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "snn_internal.cuh"

using namespace snn;

namespace {

constexpr uint64_t kMagic = 0x534e4e5354415431ull;   // "SNNSTAT1"

struct Header {
    uint64_t magic;
    uint64_t n_total;
    uint64_t n_pops;
    uint64_t n_projs;
    uint64_t shape;        // FNV-1a hash of population kinds/sizes and projection ends/sizes
};

uint64_t shape_hash(const snn_net* net) {
    uint64_t h = 1469598103934665603ull;
    auto mix = [&h](uint64_t v) {
        for (int b = 0; b < 8; ++b) {
            h ^= (v >> (8 * b)) & 0xffu;
            h *= 1099511628211ull;
        }
    };
    for (const auto& p : net->pops) { mix((uint64_t)p.d.kind); mix((uint64_t)p.d.n); }
    for (const auto& q : net->projs) { mix((uint64_t)q.d.pre); mix((uint64_t)q.d.post); mix((uint64_t)q.nnz); }
    return h;
}

struct Part {
    void* ptr;
    size_t bytes;
};

std::vector<Part> parts(snn_net* net) {
    const size_t NT = std::max<size_t>(1, (size_t)net->n_total);
    const size_t np = net->pops.size();
    return {
        {net->V, 7 * NT * sizeof(float)},            // V, m, h, n, g0, g1, I_ext (contiguous)
        {net->spk, NT * sizeof(int32_t)},
        {net->nrn_count, NT * sizeof(int32_t)},
        {net->nspk, 2 * np * sizeof(int32_t)},
        {net->counters, 2 * np * sizeof(unsigned long long)},
        {net->acc, 4 * NT * sizeof(float)},
        {net->ticket, 2 * sizeof(unsigned long long)},
        {net->bar, sizeof(GridBarrier)},
    };
}

size_t snapshot_bytes(snn_net* net) {
    size_t b = sizeof(Header);
    for (const Part& p : parts(net)) b += p.bytes;
    return b;
}

#define CK(call, what)                                     \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

snn_status copy_state(snn_net* net, void* buf, size_t bytes, int buf_is_device, bool save, cudaStream_t s) {
    if (bytes < snapshot_bytes(net)) return fail(SNN_ERR_SIZE, "snapshot buffer too small (see snn_state_size)");
    Header h{kMagic, (uint64_t)net->n_total, (uint64_t)net->pops.size(), (uint64_t)net->projs.size(),
             shape_hash(net)};
    char* p = static_cast<char*>(buf);
    const cudaMemcpyKind to_buf = buf_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const cudaMemcpyKind from_buf = buf_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (save) {
        CK(cudaMemcpyAsync(p, &h, sizeof(h), buf_is_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, s),
           "write header");
    } else {
        Header got{};
        CK(cudaMemcpyAsync(&got, p, sizeof(got), buf_is_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost, s),
           "read header");
        CK(cudaStreamSynchronize(s), "synchronize");
        if (got.magic != h.magic || got.n_total != h.n_total || got.n_pops != h.n_pops || got.n_projs != h.n_projs ||
            got.shape != h.shape)
            return fail(SNN_ERR_STATE, "snapshot was taken from a network of another shape");
    }
    p += sizeof(Header);
    for (const Part& part : parts(net)) {
        if (save) CK(cudaMemcpyAsync(p, part.ptr, part.bytes, to_buf, s), "save state");
        else CK(cudaMemcpyAsync(part.ptr, p, part.bytes, from_buf, s), "load state");
        p += part.bytes;
    }
    CK(cudaStreamSynchronize(s), "synchronize");
    return SNN_OK;
}

struct Choice {
    int32_t engine, prop_blocks, chunk, tiled;
    double us_per_step;
};

std::mutex g_cache_mu;
std::map<std::string, Choice> g_cache;

std::string shape_key(snn_net* net) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::string k = std::to_string(dev) + "|" + std::to_string(net->n_sub);
    for (const auto& p : net->pops) k += "|" + std::to_string(p.d.kind) + ":" + std::to_string(p.d.n);
    for (const auto& q : net->projs)
        k += "|" + std::to_string(q.d.pre) + ">" + std::to_string(q.d.post) + ":" + std::to_string(q.d.layout) +
             ":" + std::to_string(q.nnz);
    for (const auto& d : net->shared) k += "|shared:" + std::to_string(d.B) + "x" + std::to_string(d.n_pre);
    return k;
}

// Times one configuration on `trial_steps` steps from the snapshot `snap`
// (a warm-up run first, both from the same state); leaves the state at the
// end of the trial.
snn_status trial(snn_net* net, Choice& c, int32_t trial_steps, void* snap, size_t nb, cudaEvent_t e0, cudaEvent_t e1,
                 void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    snn_status st;
    if ((st = snn_set_option(net, SNN_OPT_ENGINE, c.engine)) != SNN_OK) return st;
    if ((st = snn_set_option(net, SNN_OPT_PROP_BLOCKS, c.prop_blocks)) != SNN_OK) return st;
    if ((st = snn_set_option(net, SNN_OPT_CHUNK, c.chunk)) != SNN_OK) return st;
    if ((st = snn_set_option(net, SNN_OPT_TILED, c.tiled)) != SNN_OK) return st;
    if ((st = snn_load_state(net, snap, nb, 1, stream)) != SNN_OK) return st;
    if ((st = snn_step(net, std::min<int64_t>(trial_steps, net->graph_steps), stream)) != SNN_OK) return st;  // warm
    if ((st = snn_load_state(net, snap, nb, 1, stream)) != SNN_OK) return st;
    cudaEventRecord(e0, s);
    if ((st = snn_step(net, trial_steps, stream)) != SNN_OK) return st;
    cudaEventRecord(e1, s);
    if ((st = snn_sync(net, stream)) != SNN_OK) return st;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    c.us_per_step = 1e3 * ms / trial_steps;
    return SNN_OK;
}

// Times the candidates from a snapshot of the live network, restores it, and
// returns the fastest in *best (options restored on failure).
snn_status time_candidates(snn_net* net, std::vector<Choice>& cands, int32_t trial_steps, Choice* best,
                           void* stream) {
    const size_t nb = snapshot_bytes(net);
    void* snap = net->mem.get(nb);
    if (!snap) return fail(SNN_ERR_OOM, "tuning snapshot");
    snn_status st = snn_save_state(net, snap, nb, 1, stream);
    const int32_t engine0 = net->engine, blocks0 = net->prop_blocks, chunk0 = net->chunk, tiled0 = net->tiled;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (st == SNN_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        st = fail(SNN_ERR_CUDA, "create events");
    best->us_per_step = 1e30;
    for (Choice& c : cands) {
        if (st != SNN_OK) break;
        if ((st = trial(net, c, trial_steps, snap, nb, e0, e1, stream)) != SNN_OK) break;
        if (c.us_per_step < best->us_per_step) *best = c;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    const snn_status rs = snn_load_state(net, snap, nb, 1, stream);
    net->mem.put(snap);
    if (st != SNN_OK) {
        net->engine = engine0; net->prop_blocks = blocks0; net->chunk = chunk0; net->tiled = tiled0;
        return st;
    }
    return rs;
}

snn_status apply(snn_net* net, const Choice& c, bool cached, snn_tuning* result) {
    snn_status st = snn_set_option(net, SNN_OPT_ENGINE, c.engine);
    if (st == SNN_OK) st = snn_set_option(net, SNN_OPT_PROP_BLOCKS, c.prop_blocks);
    if (st == SNN_OK) st = snn_set_option(net, SNN_OPT_CHUNK, c.chunk);
    if (st == SNN_OK) st = snn_set_option(net, SNN_OPT_TILED, c.tiled);
    if (st != SNN_OK) return st;
    if (result) {
        result->engine = c.engine;
        result->prop_blocks = c.prop_blocks;
        result->chunk = c.chunk;
        result->tiled = c.tiled;
        result->us_per_step = c.us_per_step;
        result->cached = cached ? 1 : 0;
    }
    return SNN_OK;
}

}  // namespace

extern "C" {

snn_status snn_state_size(snn_net* net, size_t* bytes) {
    if (!net || !bytes) return fail(SNN_ERR_INVALID_ARG, "bad argument");
    *bytes = snapshot_bytes(net);
    return SNN_OK;
}

snn_status snn_save_state(snn_net* net, void* dst, size_t bytes, int32_t dst_is_device, void* stream) {
    if (!net || !dst) return fail(SNN_ERR_INVALID_ARG, "bad argument");
    const snn_status st = snn_sync(net, stream);
    if (st != SNN_OK) return st;
    return copy_state(net, dst, bytes, dst_is_device, true, (cudaStream_t)stream);
}

snn_status snn_load_state(snn_net* net, const void* src, size_t bytes, int32_t src_is_device, void* stream) {
    if (!net || !src) return fail(SNN_ERR_INVALID_ARG, "bad argument");
    // a snapshot may hold channel-1 conductances and drive currents written
    // into the network it came from: the step kernels process them from now on
    CK(mark_state_live(net, -1, true, true, (cudaStream_t)stream), "mark state live");
    return copy_state(net, const_cast<void*>(src), bytes, src_is_device, false, (cudaStream_t)stream);
}

snn_status snn_autotune(snn_net* net, int32_t trial_steps, snn_tuning* result, void* stream) {
    if (!net || trial_steps < 1) return fail(SNN_ERR_INVALID_ARG, "bad network or trial length");
    const std::string key = shape_key(net) + "|" + std::to_string(trial_steps);
    Choice best{};
    bool cached = false;
    {
        std::lock_guard<std::mutex> lock(g_cache_mu);
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            best = it->second;
            cached = true;
        }
    }
    if (!cached) {
        std::vector<Choice> cands;
        const int sm = net->sm_count;
        // the propagation settings that give different kernels: row kernel
        // only, and the library's choice when it differs from that
        std::vector<int> tileds{0};
        if (propagation_modes(net, 2) != propagation_modes(net, 0)) tileds.push_back(2);
        for (int blocks : {2 * sm, 4 * sm, 8 * sm})
            for (int chunk : {512, 1024, 2048})
                for (int tiled : tileds) cands.push_back({0, blocks, chunk, tiled, 0.0});
        // shared dense projections step in the plain engine only
        if (net->persist_grid > 0 && net->shared.empty()) cands.push_back({1, 4 * sm, 1024, 2, 0.0});
        if (net->cluster_size > 0 && net->shared.empty()) cands.push_back({3, 4 * sm, 1024, 2, 0.0});
        const snn_status st = time_candidates(net, cands, trial_steps, &best, stream);
        if (st != SNN_OK) return st;
        std::lock_guard<std::mutex> lock(g_cache_mu);
        g_cache[key] = best;
    }
    return apply(net, best, cached, result);
}

snn_status snn_occupancy_config(snn_net* net, int32_t trial_steps, snn_tuning* result, void* stream) {
    if (!net || trial_steps < 1) return fail(SNN_ERR_INVALID_ARG, "bad network or trial length");
    if (net->graded) return fail(SNN_ERR_STATE, "graded networks have no launch options");
    // Sec. 3's rule: the two-kernel step with each kernel's grid filled to its
    // occupancy limit (resident blocks per SM x SMs); no measurement involved.
    int per_sm = 0;
    const cudaError_t e = propagate_occupancy(&per_sm);
    if (e != cudaSuccess) return cuda_fail(e, "propagation occupancy");
    std::vector<Choice> one{{0, std::max(1, per_sm) * net->sm_count, 1024, 0, 0.0}};
    Choice c{};
    const snn_status st = time_candidates(net, one, trial_steps, &c, stream);
    if (st != SNN_OK) return st;
    return apply(net, c, false, result);
}

}  // extern "C"
