// Host side of the differentiable (graded-synapse) form: creation-time
// transposed copies of the compressed rows, plain stepping, the recorded
// forward with checkpoints every K steps, and the adjoint sweep that
// recomputes each segment from its checkpoint.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "snn_internal.cuh"

using namespace snn;

namespace snn {

bool graded_requested(const snn_proj_desc* projs, int n_projs) {
    for (int q = 0; q < n_projs; ++q)
        if (projs[q].synapse == SNN_SYN_GRADED) return true;
    return false;
}

namespace {

GradedArgs graded_args(snn_net* net) {
    GradedArgs a{};
    a.pops = net->d_pops;
    a.tile_pop = net->tile_pop;
    a.gprojs = net->d_gprojs;
    a.n_gprojs = (int32_t)net->projs.size();
    a.total_posts = net->total_posts;
    a.spmv_items = net->spmv_items;
    a.in_begin = net->in_begin;
    a.in_list = net->in_list;
    a.out_begin = net->out_begin;
    a.out_list = net->out_list;
    a.n_total = net->n_total;
    a.narrow = net->graded_narrow ? 1 : 0;
    a.V = net->V; a.m = net->m; a.h = net->h; a.n = net->n; a.iext = net->iext;
    a.r = net->r;
    a.G = net->G;
    a.y = net->y;
    a.out_pop = net->rec_out_pop;
    a.n_out = net->rec_n_out;
    a.n_sub = net->n_sub;
    a.hs = (float)(net->dt / net->n_sub);
    a.a_filter = net->rec_tau > 0 ? (float)(net->dt / net->rec_tau) : 0.0f;
    a.seed_lo = (uint32_t)net->seed;
    a.seed_hi = (uint32_t)(net->seed >> 32);
    return a;
}

// One time step: graded conductances from the current releases (the sparse
// projections in one launch, each dense projection in its own), then the
// neuron update.  `G` receives the step's G vector.
cudaError_t graded_one_step(snn_net* net, GradedArgs a, float* G, int64_t t, cudaStream_t s) {
    a.G = G;
    a.t_rng = (uint32_t)t;
    cudaError_t e = launch_graded_spmv(a, s);
    for (size_t q = 0; q < net->projs.size() && e == cudaSuccess; ++q) {
        const ProjHost& P = net->projs[q];
        if (P.d.layout != SNN_LAYOUT_DENSE) continue;
        const PopHost& pre = net->pops[P.d.pre];
        e = launch_graded_dense_fwd(P.w, a.r + pre.offset, pre.d.n, net->pops[P.d.post].d.n, G + P.g_off, P.dpart,
                                    P.dld, P.dcount, P.dchunks, P.dstream, s);
    }
    if (e == cudaSuccess) e = launch_graded_neuron(a, s);
    return e;
}

snn_status upload_gprojs(snn_net* net) {
    std::vector<GradProj> g(net->projs.size());
    int64_t items = 0;
    for (size_t q = 0; q < g.size(); ++q) {
        const ProjHost& P = net->projs[q];
        const PopHost& pre = net->pops[P.d.pre];
        const PopHost& post = net->pops[P.d.post];
        GradProj& d = g[q];
        d.pre = P.d.pre;
        d.post = P.d.post;
        d.pre_off = pre.offset;
        d.post_off = post.offset;
        d.n_pre = pre.d.n;
        d.n_post = post.d.n;
        d.scale = P.scale;
        d.E = (float)post.d.E_syn[P.d.channel];
        d.g_off = P.g_off;
        d.row_ptr = P.row_ptr;
        d.col = P.col;
        d.col16 = P.col16;
        d.w = P.w;
        d.csc_ptr = P.csc_ptr;
        d.csc_pre = P.csc_pre;
        d.csc_pre16 = P.csc_pre16;
        d.csc_w = P.csc_w;
        d.dense = P.d.layout == SNN_LAYOUT_DENSE ? 1 : 0;
        // forward product: posts with short transposed rows (fewer than 24
        // synapses on average) one per lane, 32 to a work item; longer rows
        // one post per warp; dense storage has its own product
        d.lane_rows = (!d.dense && (double)P.nnz < 24.0 * std::max(1, d.n_post)) ? 1 : 0;
        d.item_off = items;
        if (!d.dense) items += d.lane_rows ? (d.n_post + 31) / 32 : d.n_post;
    }
    net->spmv_items = items;
    if (!g.empty())
        SNN_CK(cudaMemcpy(net->d_gprojs, g.data(), g.size() * sizeof(GradProj), cudaMemcpyHostToDevice),
               "upload graded projections");
    return SNN_OK;
}

}  // namespace

// Called by create_impl for graded networks, after the compressed rows are
// validated and stored: transposed copies, per-population lists, releases.
snn_status graded_setup(snn_net* net, cudaStream_t s) {
    const int np = (int)net->pops.size(), nq = (int)net->projs.size();
    if (nq > kMaxGradedProjs) return fail(SNN_ERR_INVALID_ARG, "at most 64 graded projections");
    if (net->n_sub > kMaxSub) return fail(SNN_ERR_INVALID_ARG, "graded networks take at most 16 substeps");
    net->graded = true;
    // release parameters per pre population: shared by all its outgoing projections
    std::vector<double> thr((size_t)np, -20.0), slope((size_t)np, 2.0);
    std::vector<int> seen((size_t)np, 0);
    for (int q = 0; q < nq; ++q) {
        const snn_proj_desc& d = net->projs[q].d;
        if (d.synapse != SNN_SYN_GRADED)
            return fail(SNN_ERR_INVALID_ARG, "a graded network takes only graded projections");
        if (!(d.v_slope > 0) || !std::isfinite(d.v_thr))
            return fail(SNN_ERR_INVALID_ARG, "graded projection needs v_slope > 0 and finite v_thr");
        if (seen[d.pre] && (thr[d.pre] != d.v_thr || slope[d.pre] != d.v_slope))
            return fail(SNN_ERR_INVALID_ARG, "projections leaving one population must share v_thr and v_slope");
        seen[d.pre] = 1;
        thr[d.pre] = d.v_thr;
        slope[d.pre] = d.v_slope;
    }
    for (int k = 0; k < np; ++k)
        if (net->pops[k].d.kind != SNN_POP_HH) return fail(SNN_ERR_INVALID_ARG, "graded networks take HH populations");
    // transposed copies, built on the host with a stable counting sort so that
    // each post's entries stay in ascending pre order (deterministic sums)
    net->graded_narrow = true;
    for (int q = 0; q < nq; ++q)
        if (net->pops[net->projs[q].d.pre].d.n > 65536) net->graded_narrow = false;
    int64_t g_off = 0;
    for (int q = 0; q < nq; ++q) {
        ProjHost& P = net->projs[q];
        const int32_t n_pre = net->pops[P.d.pre].d.n, n_post = net->pops[P.d.post].d.n;
        if (P.d.layout == SNN_LAYOUT_DENSE) {
            // the matrix itself serves both directions; the forward product's
            // partial rows and per post block tickets
            P.dchunks = dense_fwd_chunks(n_pre, n_post, net->sm_count);
            // a matrix within 60 % of L2 stays resident from step to step
            P.dstream = 4.0 * (double)n_pre * (double)n_post > 0.6 * (double)net->l2_bytes;
            P.dld = ((int64_t)n_post + 3) / 4 * 4;
            const size_t blocks = ((size_t)n_post + 127) / 128;
            SNN_TRY(net_alloc(net, &P.dpart, std::max<size_t>(1, (size_t)P.dchunks * P.dld), "dense partial rows"));
            SNN_TRY(net_alloc(net, &P.dcount, std::max<size_t>(1, blocks), "dense tickets"));
            SNN_CK(cudaMemsetAsync(P.dcount, 0, std::max<size_t>(1, blocks) * sizeof(unsigned), s), "clear");
            P.g_off = g_off;
            g_off += n_post;
            continue;
        }
        std::vector<int64_t> rp((size_t)n_pre + 1);
        std::vector<int32_t> col((size_t)P.nnz);
        std::vector<float> w((size_t)P.nnz);
        SNN_CK(cudaMemcpyAsync(rp.data(), P.row_ptr, rp.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, s), "rows");
        if (P.nnz) {
            SNN_CK(cudaMemcpyAsync(col.data(), P.col, col.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, s), "cols");
            SNN_CK(cudaMemcpyAsync(w.data(), P.w, w.size() * sizeof(float), cudaMemcpyDeviceToHost, s), "weights");
        }
        SNN_CK(cudaStreamSynchronize(s), "synchronize");
        std::vector<int64_t> cp((size_t)n_post + 1, 0);
        for (int64_t e = 0; e < P.nnz; ++e) cp[(size_t)col[e] + 1]++;
        for (int32_t j = 0; j < n_post; ++j) cp[(size_t)j + 1] += cp[j];
        std::vector<int64_t> pos(cp.begin(), cp.end() - 1), perm((size_t)P.nnz);
        std::vector<int32_t> cpre((size_t)P.nnz);
        std::vector<float> cw((size_t)P.nnz);
        for (int32_t i = 0; i < n_pre; ++i)
            for (int64_t e = rp[i]; e < rp[(size_t)i + 1]; ++e) {
                const int64_t k = pos[col[e]]++;
                cpre[k] = i;
                cw[k] = w[e];
                perm[k] = e;
            }
        SNN_TRY(net_alloc(net, &P.csc_ptr, (size_t)n_post + 1, "transposed row starts"));
        // padded to a multiple of 4 plus 4 zeros, so 16-byte loads that start
        // at or before a column's end stay inside the allocation
        const size_t padded = (size_t)((P.nnz + 3) / 4 * 4 + 4);
        // pre indices in 16 bits when every graded pre population allows
        // (the sparse product then streams 6 instead of 8 bytes per synapse)
        const bool narrow = net->graded_narrow;
        if (narrow) {
            SNN_TRY(net_alloc(net, &P.csc_pre16, padded, "transposed indices"));
            SNN_CK(cudaMemsetAsync(P.csc_pre16, 0, padded * sizeof(uint16_t), s), "clear");
        } else {
            SNN_TRY(net_alloc(net, &P.csc_pre, padded, "transposed indices"));
            SNN_CK(cudaMemsetAsync(P.csc_pre, 0, padded * sizeof(int32_t), s), "clear");
        }
        SNN_TRY(net_alloc(net, &P.csc_w, padded, "transposed weights"));
        SNN_CK(cudaMemsetAsync(P.csc_w, 0, padded * sizeof(float), s), "clear");
        SNN_TRY(net_alloc(net, &P.csc_perm, std::max<size_t>(1, (size_t)P.nnz), "transposed positions"));
        SNN_CK(cudaMemcpyAsync(P.csc_ptr, cp.data(), cp.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s), "upload");
        if (P.nnz) {
            if (narrow) {
                std::vector<uint16_t> c16(cpre.begin(), cpre.end());
                SNN_CK(cudaMemcpyAsync(P.csc_pre16, c16.data(), c16.size() * sizeof(uint16_t), cudaMemcpyHostToDevice, s),
                       "upload");
                SNN_CK(cudaStreamSynchronize(s), "synchronize");      // c16 leaves scope
            } else {
                SNN_CK(cudaMemcpyAsync(P.csc_pre, cpre.data(), cpre.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                                       s), "upload");
            }
            SNN_CK(cudaMemcpyAsync(P.csc_w, cw.data(), cw.size() * sizeof(float), cudaMemcpyHostToDevice, s), "upload");
            SNN_CK(cudaMemcpyAsync(P.csc_perm, perm.data(), perm.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s),
                   "upload");
        }
        // the adjoint gather streams the compressed rows: their post indices in
        // 16 bits when the post population allows (6 instead of 8 bytes per synapse)
        if (n_post <= 65536 && P.nnz) {
            // padded like the weights (a multiple of 4 plus 4), so 8-byte loads of
            // four indices that start before a row's end stay inside the allocation
            const size_t padded16 = (size_t)((P.nnz + 3) / 4 * 4 + 4);
            SNN_TRY(net_alloc(net, &P.col16, padded16, "16-bit post indices"));
            std::vector<uint16_t> c16(padded16, 0);
            std::copy(col.begin(), col.end(), c16.begin());
            SNN_CK(cudaMemcpyAsync(P.col16, c16.data(), c16.size() * sizeof(uint16_t), cudaMemcpyHostToDevice, s),
                   "upload");
            SNN_CK(cudaStreamSynchronize(s), "synchronize");      // c16 leaves scope
        }
        SNN_CK(cudaStreamSynchronize(s), "synchronize");
        P.g_off = g_off;
        g_off += n_post;
    }
    net->total_posts = g_off;
    // incoming projections per population
    std::vector<int32_t> ib((size_t)np + 1, 0), il;
    for (int k = 0; k < np; ++k) {
        ib[k] = (int32_t)il.size();
        for (int q = 0; q < nq; ++q)
            if (net->projs[q].d.post == k) il.push_back(q);
    }
    ib[np] = (int32_t)il.size();
    if (il.empty()) il.push_back(0);
    const size_t NT = std::max<size_t>(1, (size_t)net->n_total);
    SNN_TRY(net_alloc(net, &net->d_gprojs, std::max<size_t>(1, (size_t)nq), "graded projections"));
    SNN_TRY(net_alloc(net, &net->in_begin, (size_t)np + 1, "incoming offsets"));
    SNN_TRY(net_alloc(net, &net->in_list, il.size(), "incoming projections"));
    SNN_TRY(net_alloc(net, &net->r, NT, "releases"));
    SNN_TRY(net_alloc(net, &net->G, std::max<size_t>(1, (size_t)g_off), "graded conductances"));
    SNN_TRY(net_alloc(net, &net->y, NT, "output filter"));
    SNN_TRY(net_alloc(net, &net->d_grad_scale, std::max<size_t>(1, (size_t)nq), "scale gradients"));
    SNN_CK(cudaMemcpyAsync(net->in_begin, ib.data(), ib.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s), "upload");
    SNN_CK(cudaMemcpyAsync(net->in_list, il.data(), il.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s), "upload");
    SNN_CK(cudaMemsetAsync(net->y, 0, NT * sizeof(float), s), "clear");
    SNN_CK(cudaStreamSynchronize(s), "synchronize");
    // release parameters into the population descriptors
    std::vector<DevPop> dp((size_t)np);
    SNN_CK(cudaMemcpy(dp.data(), net->d_pops, dp.size() * sizeof(DevPop), cudaMemcpyDeviceToHost), "read pops");
    for (int k = 0; k < np; ++k) {
        dp[k].rel_thr = (float)thr[k];
        dp[k].rel_inv_slope = (float)(1.0 / slope[k]);
    }
    SNN_CK(cudaMemcpy(net->d_pops, dp.data(), dp.size() * sizeof(DevPop), cudaMemcpyHostToDevice), "write pops");
    SNN_TRY(upload_gprojs(net));
    return graded_reset(net, s);
}

// Releases from the current V; the output filter starts at the output V.
snn_status graded_reset(snn_net* net, cudaStream_t s) {
    net->g_t = 0;
    GradedArgs a = graded_args(net);
    SNN_CK(launch_graded_release_init(a, s), "initial releases");
    return SNN_OK;
}

snn_status graded_step(snn_net* net, int64_t n_steps, cudaStream_t s) {
    GradedArgs a = graded_args(net);
    a.out_pop = -1;
    for (int64_t k = 0; k < n_steps; ++k) {
        SNN_CK(graded_one_step(net, a, net->G, net->g_t, s), "graded step");
        ++net->g_t;
    }
    return SNN_OK;
}

}  // namespace snn

namespace {

snn_status ensure_segment_buffers(snn_net* net, int32_t K, int32_t n_out) {
    if (net->seg_cap_K >= K) return SNN_OK;
    const size_t NT = std::max<size_t>(1, (size_t)net->n_total), G = std::max<int64_t>(1, net->total_posts);
    const size_t kp = ((size_t)K + 3) / 4 * 4;
    SNN_TRY(net_alloc(net, &net->seg_state, (size_t)K * 5 * NT, "segment states"));
    SNN_TRY(net_alloc(net, &net->seg_r, (size_t)K * NT, "segment releases"));
    SNN_TRY(net_alloc(net, &net->seg_G, (size_t)K * G, "segment conductances"));
    SNN_TRY(net_alloc(net, &net->nu_step, G, "step dL/dG"));
    SNN_TRY(net_alloc(net, &net->nu_km, G * kp, "segment dL/dG"));
    SNN_TRY(net_alloc(net, &net->adj, 6 * NT, "adjoints"));
    // operand parts of the tensor-core weight gradient, sized for the largest dense projection
    size_t need_a = 0, need_b = 0;
    for (const auto& P : net->projs) {
        if (P.d.layout != SNN_LAYOUT_DENSE) continue;
        int64_t mp, np, kpg;
        dense_grad_sizes(net->pops[P.d.pre].d.n, net->pops[P.d.post].d.n, K, &mp, &np, &kpg);
        need_a = std::max(need_a, (size_t)(3 * mp * kpg));
        need_b = std::max(need_b, (size_t)(3 * np * kpg));
    }
    if (need_a > net->grad_A_cap) {
        SNN_TRY(net_alloc(net, &net->grad_A, need_a, "gradient operand parts"));
        net->grad_A_cap = need_a;
    }
    if (need_b > net->grad_B_cap) {
        SNN_TRY(net_alloc(net, &net->grad_B, need_b, "gradient operand parts"));
        net->grad_B_cap = need_b;
    }
    (void)n_out;
    net->seg_cap_K = K;
    return SNN_OK;
}

}  // namespace

extern "C" {

snn_status snn_set_scale(snn_net* net, int32_t proj, double scale) {
    if (!net || proj < 0 || proj >= (int32_t)net->projs.size() || !std::isfinite(scale))
        return fail(SNN_ERR_INVALID_ARG, "bad projection or scale");
    net->projs[proj].scale = (float)scale;
    snn_status st = SNN_OK;
    if (net->graded) st = upload_gprojs(net);
    if (st != SNN_OK) return st;
    // spiking networks: projection descriptors and any captured graph
    return snn_set_option(net, SNN_OPT_CHUNK, net->chunk);
}

snn_status snn_set_weights(snn_net* net, int32_t proj, const float* w, int32_t on_device, void* stream) {
    if (!net || !w || proj < 0 || proj >= (int32_t)net->projs.size()) return fail(SNN_ERR_INVALID_ARG, "bad argument");
    ProjHost& P = net->projs[proj];
    cudaStream_t s = (cudaStream_t)stream;
    // compressed rows: nnz weights in row order; dense storage: the n_pre x n_post matrix
    if (P.nnz)
        SNN_CK(cudaMemcpyAsync(P.w, w, sizeof(float) * P.nnz, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                               s), "copy weights");
    if (net->graded && P.d.layout == SNN_LAYOUT_CSR)
        SNN_CK(launch_scatter_csc(P.w, P.csc_perm, P.csc_w, P.nnz, s), "transposed weights");
    SNN_CK(cudaStreamSynchronize(s), "synchronize");
    return SNN_OK;
}

snn_status snn_graded_launch_product(snn_net* net, void* stream) {
    if (!net) return fail(SNN_ERR_INVALID_ARG, "net is NULL");
    if (!net->graded) return fail(SNN_ERR_STATE, "not a graded network");
    GradedArgs a = graded_args(net);
    SNN_CK(launch_graded_spmv(a, (cudaStream_t)stream), "graded product");
    return SNN_OK;
}

snn_status snn_forward_record(snn_net* net, int64_t n_steps, int32_t checkpoint_every, int32_t out_pop,
                              double tau_f, float* y_out, void* stream) {
    if (!net) return fail(SNN_ERR_INVALID_ARG, "net is NULL");
    if (!net->graded) return fail(SNN_ERR_STATE, "recorded forward needs a graded network");
    if (n_steps < 1 || n_steps >= (int64_t(1) << 31) || checkpoint_every < 1 || checkpoint_every > kMaxSeg ||
        out_pop < 0 || out_pop >= (int32_t)net->pops.size() || !(tau_f > 0) || !y_out)
        return fail(SNN_ERR_INVALID_ARG, "bad steps, checkpoint interval (1..512), output population, tau or y_out");
    cudaStream_t s = (cudaStream_t)stream;
    const int32_t n_out = net->pops[out_pop].d.n;
    const size_t NT = std::max<size_t>(1, (size_t)net->n_total);
    const int64_t n_ckpt = (n_steps + checkpoint_every - 1) / checkpoint_every;
    // checkpoint buffer (grown as needed)
    if (net->rec_ckpt_cap < (size_t)n_ckpt * 6 * NT) {
        SNN_TRY(net_alloc(net, &net->rec_ckpt, (size_t)n_ckpt * 6 * NT, "checkpoints"));
        net->rec_ckpt_cap = (size_t)n_ckpt * 6 * NT;
    }
    SNN_TRY(ensure_segment_buffers(net, checkpoint_every, n_out));
    // the whole trajectory (step-start states, releases, G) when it takes at
    // most a quarter of the free device memory: snn_backward then reads it
    // instead of recomputing every checkpoint segment
    const size_t G = std::max<int64_t>(1, net->total_posts);
    bool store = false;
    if (net->graded_store) {
        size_t free_b = 0, total_b = 0;
        store = cudaMemGetInfo(&free_b, &total_b) == cudaSuccess &&
                (double)n_steps * (double)(6 * NT + G) * sizeof(float) <= 0.25 * (double)free_b;
        if (store && net->traj_cap_steps < (size_t)n_steps) {
            store = net_alloc(net, &net->traj_state, (size_t)n_steps * 5 * NT, "trajectory states") == SNN_OK &&
                    net_alloc(net, &net->traj_r, (size_t)n_steps * NT, "trajectory releases") == SNN_OK &&
                    net_alloc(net, &net->traj_G, (size_t)n_steps * G, "trajectory conductances") == SNN_OK;
            net->traj_cap_steps = store ? (size_t)n_steps : 0;
        }
    }
    net->rec_stored = store;
    net->rec_T = n_steps;
    net->rec_K = checkpoint_every;
    net->rec_out_pop = out_pop;
    net->rec_n_out = n_out;
    net->rec_tau = tau_f;
    // start from the creation state
    SNN_TRY(snn_reset(net, stream));
    GradedArgs a = graded_args(net);
    a.y_out = y_out;
    SNN_TRY(graded_reset(net, s));
    for (int64_t t = 0; t < n_steps; ++t) {
        float* Gt = net->G;
        if (store) {
            a.rec_state = net->traj_state + (size_t)t * 5 * NT;
            a.rec_r = net->traj_r + (size_t)t * NT;
            Gt = net->traj_G + (size_t)t * G;
        } else if (t % checkpoint_every == 0) {
            float* c = net->rec_ckpt + (size_t)(t / checkpoint_every) * 6 * NT;
            SNN_CK(cudaMemcpyAsync(c, net->V, 4 * NT * sizeof(float), cudaMemcpyDeviceToDevice, s), "checkpoint");
            SNN_CK(cudaMemcpyAsync(c + 4 * NT, net->iext, NT * sizeof(float), cudaMemcpyDeviceToDevice, s), "checkpoint");
            SNN_CK(cudaMemcpyAsync(c + 5 * NT, net->y, NT * sizeof(float), cudaMemcpyDeviceToDevice, s), "checkpoint");
        }
        a.t_rec = (int32_t)t;
        SNN_CK(graded_one_step(net, a, Gt, t, s), "recorded step");
    }
    net->g_t = n_steps;
    SNN_CK(cudaStreamSynchronize(s), "synchronize");
    return snn_sync(net, stream);
}

snn_status snn_backward(snn_net* net, const float* dL_dy, float* grad_scale, float* const* grad_w, void* stream) {
    if (!net) return fail(SNN_ERR_INVALID_ARG, "net is NULL");
    if (!net->graded || net->rec_T == 0) return fail(SNN_ERR_STATE, "no recorded forward");
    if (!dL_dy || !grad_scale || !grad_w) return fail(SNN_ERR_INVALID_ARG, "dL/dy or gradient buffers are NULL");
    const int nq = (int)net->projs.size();
    for (int q = 0; q < nq; ++q)
        if (!grad_w[q] && net->projs[q].nnz) return fail(SNN_ERR_INVALID_ARG, "weight gradient buffer is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t NT = std::max<size_t>(1, (size_t)net->n_total);
    const size_t G = std::max<int64_t>(1, net->total_posts);
    const int64_t T = net->rec_T;
    const int32_t K = net->rec_K, n_out = net->rec_n_out;
    const int32_t kp = (K + 3) / 4 * 4;
    for (int q = 0; q < nq; ++q)
        if (net->projs[q].nnz) SNN_CK(cudaMemsetAsync(grad_w[q], 0, sizeof(float) * net->projs[q].nnz, s), "clear");
    SNN_CK(cudaMemsetAsync(net->d_grad_scale, 0, sizeof(double) * std::max(1, nq), s), "clear");
    SNN_CK(cudaMemsetAsync(net->adj, 0, 6 * NT * sizeof(float), s), "clear adjoints");
    AdjArgs b{};
    b.lV = net->adj;
    b.lV_loc = net->adj + NT;
    b.lm = net->adj + 2 * NT;
    b.lh = net->adj + 3 * NT;
    b.ln = net->adj + 4 * NT;
    b.ly = net->adj + 5 * NT;
    b.nu_step = net->nu_step;
    b.nu_km = net->nu_km;
    b.kp = kp;
    b.grad_scale = net->d_grad_scale;
    const int64_t n_seg = (T + K - 1) / K;
    const bool stored = net->rec_stored;
    for (int64_t seg = n_seg - 1; seg >= 0; --seg) {
        const int64_t t0 = seg * K;
        const int32_t L = (int32_t)std::min<int64_t>(K, T - t0);
        // the segment's step-start states, releases and G: kept by the
        // recorded forward, or recomputed from the segment's checkpoint
        float* seg_state = stored ? net->traj_state + (size_t)t0 * 5 * NT : net->seg_state;
        float* seg_r = stored ? net->traj_r + (size_t)t0 * NT : net->seg_r;
        float* seg_G = stored ? net->traj_G + (size_t)t0 * G : net->seg_G;
        b.r_seg = seg_r;
        GradedArgs a = graded_args(net);
        if (!stored) {
            const float* c = net->rec_ckpt + (size_t)seg * 6 * NT;
            SNN_CK(cudaMemcpyAsync(net->V, c, 4 * NT * sizeof(float), cudaMemcpyDeviceToDevice, s), "restore");
            SNN_CK(cudaMemcpyAsync(net->iext, c + 4 * NT, NT * sizeof(float), cudaMemcpyDeviceToDevice, s), "restore");
            SNN_CK(cudaMemcpyAsync(net->y, c + 5 * NT, NT * sizeof(float), cudaMemcpyDeviceToDevice, s), "restore");
            // releases from the restored V, without resetting the filter
            GradedArgs ri = a;
            ri.out_pop = -1;
            SNN_CK(launch_graded_release_init(ri, s), "segment releases");
            for (int32_t tl = 0; tl < L; ++tl) {
                GradedArgs f = a;
                f.rec_state = seg_state + (size_t)tl * 5 * NT;
                f.rec_r = seg_r + (size_t)tl * NT;
                f.t_rec = (int32_t)(t0 + tl);
                SNN_CK(graded_one_step(net, f, seg_G + (size_t)tl * G, t0 + tl, s), "segment recompute");
            }
        }
        // reverse sweep over the segment
        for (int32_t tl = L - 1; tl >= 0; --tl) {
            GradedArgs r = a;
            r.G = seg_G + (size_t)tl * G;
            r.dL_dy = dL_dy;
            r.t_rec = (int32_t)(t0 + tl);
            b.st = seg_state + (size_t)tl * 5 * NT;
            b.r_step = seg_r + (size_t)tl * NT;
            b.tl = tl;
            SNN_CK(launch_graded_reverse(r, b, s), "reverse step");
        }
        for (int q = 0; q < nq; ++q) {
            const ProjHost& P = net->projs[q];
            if (P.d.layout == SNN_LAYOUT_DENSE) {
                DenseGradArgs g{};
                g.R = seg_r + net->pops[P.d.pre].offset;          // releases of the pre population
                g.ldr = (int64_t)NT;
                g.N = net->nu_km + (size_t)P.g_off * kp;           // dL/dG of the projection's posts
                g.ldn = kp;
                g.m = net->pops[P.d.pre].d.n;
                g.n = net->pops[P.d.post].d.n;
                g.L = L;
                g.D = grad_w[q];
                g.ldd = g.n;
                g.engine = net->dense_grad;
                g.A = net->grad_A;
                g.B = net->grad_B;
                g.error = net->error;
                g.spin_limit = net->spin_limit;
                SNN_CK(launch_dense_grad(g, s), "dense weight gradients");
            } else {
                SNN_CK(launch_graded_sddmm(a, b, q, net->pops[P.d.pre].d.n, grad_w[q], L, s), "weight gradients");
            }
        }
    }
    SNN_CK(launch_finish_grad_scale(net->d_grad_scale, grad_scale, nq, s), "scale gradients");
    SNN_CK(cudaStreamSynchronize(s), "synchronize");
    return snn_sync(net, stream);
}

}  // extern "C"
