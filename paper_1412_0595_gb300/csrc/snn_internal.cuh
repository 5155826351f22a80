// Internal declarations of the GB300 spiking-network library: device-side
// descriptors, the network object and the kernel launchers shared by the
// translation units.  Not part of the public C-ABI (include/snn.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "snn.h"

namespace snn {

constexpr int kTile = 256;                 // neurons per compaction tile (one CTA)
constexpr int kMaxPops = 4096;
constexpr int kMaxProjs = 4096;

// Sticky device error bits.
constexpr uint32_t kDevErrTimeout = 1u;
constexpr uint32_t kDevErrCsr = 2u;

// Philox stream identifiers (counter word 3).
constexpr uint32_t kStreamSource = 1u;
constexpr uint32_t kStreamDrive = 2u;
constexpr uint32_t kStreamCsr = 3u;
constexpr uint32_t kStreamIzhParam = 5u;        // per-neuron parameter draw r
constexpr uint32_t kStreamIzhNoise = 6u;        // 6, 7, 8: the 12 words of the input noise


struct DevPop {
    int32_t kind;          // SNN_POP_HH or SNN_POP_SOURCE
    int32_t n;
    int32_t offset;        // first index in the SoA state arrays (multiple of kTile)
    int32_t first_tile;    // first compaction tile
    int32_t n_tiles;
    uint32_t tag;          // RNG tag (instance << 8 | population index mod 256 within instance)
    float gNa, ENa, gK, EK, gL, EL;
    float hs_over_C;       // substep length / C
    float E0, E1;          // channel reversal potentials
    float d0, d1;          // channel decay factors exp(-dt / tau)
    float v_thresh;
    float drive_amp, drive_dec;
    unsigned long long thr_src;    // Bernoulli thresholds round(p * 2^32)
    unsigned long long thr_drive;
    int32_t* spk;          // spike list of the last step (ascending within each tile)
    int32_t* nspk;         // [2] list lengths, slot e & 1 for step epoch e
    unsigned long long* spike_count;
    unsigned long long* nan_count;
    int32_t* neuron_spikes;        // per-neuron spike counts of this population
    float rel_thr, rel_inv_slope;  // graded release of this population's neurons
    float izh[8];                  // Izhikevich: a0, a1, b0, b1, c0, c2, d0, d2
    float noise, bias;             // Izhikevich input: bias + noise * z
    float dt;                      // step length (ms), for u
    int32_t g1_live;               // channel 1 can be nonzero (a projection targets it, or it was written)
    int32_t iext_live;             // the drive current can be nonzero (driven, or written)
};

struct DevProj {
    int32_t layout;        // SNN_LAYOUT_CSR / SNN_LAYOUT_DENSE
    int32_t n_pre, n_post;
    int32_t chunks;        // work items per spiking row (CSR) or per row block (dense)
    float scale;
    const int64_t* row_ptr;
    const int32_t* col;
    const float* w;        // nnz (CSR) or n_pre * n_post (dense)
    float* g;              // post conductance channel, already offset to the post population
    const int32_t* spk;    // pre spike list
    const int32_t* nspk;   // [2] list lengths of the pre population (slot e & 1)
    const int32_t* pre_count;   // per-neuron spike counts of the pre population
    float* acc;            // persistent engine: event accumulator (buffer 0), offset to the post population
    int32_t post_soa;      // SoA offset of the post population
    int32_t channel;       // post conductance channel
    int32_t mode;          // compressed rows: 0 warp per row chunk, 1 post-tiled bulk copies, 2 post-tiled segments
    int32_t n_ptiles;      // post tiles of the post-tiled mode
    int32_t ptile;         // posts per tile
    const int64_t* split;  // [n_pre][n_ptiles + 1] first synapse of each row in each post tile
    const int64_t* csplit; // cluster engine: [n_pre][cluster size + 1] first synapse of each row in each CTA slice
};

// Grid barrier of the persistent engine: a monotone arrival counter.  A launch
// reads `base` once; barrier k of that launch completes when count reaches
// base + (k + 1) * gridDim.x; block 0 advances base when the launch ends.
struct GridBarrier {
    unsigned long long count;
    unsigned long long base;
};

constexpr int kMaxGradedProjs = 64;
constexpr int kMaxSub = 16;            // substeps the adjoint recomputes in registers
constexpr int kMaxSeg = 512;           // steps per checkpoint segment

struct GradProj {
    int32_t pre, post;
    int32_t pre_off, post_off;         // SoA offsets of the pre / post populations
    int32_t n_pre, n_post;
    float scale;                       // s_q
    float E;                           // reversal potential of the post channel
    int64_t g_off;                     // block of this projection in a step's G vector
    const int64_t* row_ptr;            // compressed rows (pre-major)
    const int32_t* col;
    const uint16_t* col16;             // the post indices in 16 bits when the post population has at most 65,536 neurons, else null
    const float* w;
    const int64_t* csc_ptr;            // transposed copy (post-major)
    const int32_t* csc_pre;            // pre indices, 32-bit, or
    const uint16_t* csc_pre16;         // 16-bit when every graded pre population has at most 65,536 neurons
    const float* csc_w;
    int32_t dense;                     // 1: w is the n_pre x n_post matrix (no row / column arrays)
    int32_t lane_rows;                 // forward product: 1 one post per lane (short rows), 0 one post per warp
    int64_t item_off;                  // first work item of this projection in the forward product
};

struct GradedArgs {
    const DevPop* pops;
    const int32_t* tile_pop;
    const GradProj* gprojs;
    int32_t n_gprojs;
    int64_t total_posts;               // sum of n_post over projections (length of G)
    int64_t spmv_items;                // work items of the compressed-row forward product
    const int32_t* in_begin;           // [n_pops + 1] incoming projections per population
    const int32_t* in_list;
    const int32_t* out_begin;          // [n_pops + 1] outgoing projections per population
    const int32_t* out_list;
    int32_t n_total;
    int32_t narrow;                    // transposed pre indices are 16-bit (csc_pre16)
    float *V, *m, *h, *n, *iext;
    float* r;                          // release of every neuron (next step's input)
    float* G;                          // G vector of the current step
    float* y;                          // output filter state [n_out]
    float* y_out;                      // [T][n_out] record of y (recorded forward) or nullptr
    const float* dL_dy;                // [T][n_out] caller's dL/dy (reverse sweep)
    int32_t out_pop, n_out;
    int32_t t_rec;                     // step index within the recorded forward
    uint32_t t_rng;                    // step counter of the drive random numbers
    int32_t n_sub;
    float hs, a_filter;
    uint32_t seed_lo, seed_hi;
    float* rec_state;                  // [5][n_total] step-start V, m, h, n, I_ext (after drive) or nullptr
    float* rec_r;                      // [n_total] releases used by the step
};

struct AdjArgs {
    const float* st;                   // [5][n_total] step-start state of the step being reversed
    const float* r_step;               // [n_total] releases of that step
    const float* r_seg;                // [K][n_total] releases of the segment
    float *lV, *lV_loc, *lm, *lh, *ln, *ly;
    float* nu_step;                    // [G] dL/dG of the step
    float* nu_km;                      // [G][kp] dL/dG of the segment, time-contiguous
    int32_t kp, tl;
    double* grad_scale;
};

// One rank-L update D[i][j] += sum_{t < L} R[t][i] N[j][t] (i < m, j < n):
// the weight gradient of a dense graded projection over a segment, with R
// the segment's releases of the pre population and N its dL/dG.
struct DenseGradArgs {
    const float* R;                    // R[t * ldr + i]
    int64_t ldr;
    const float* N;                    // N[j * ldn + t]
    int64_t ldn;
    int32_t m, n, L;
    float* D;                          // D[i * ldd + j]
    int64_t ldd;
    int32_t engine;                    // 0 CUDA cores, 1 tensor cores
    uint16_t *A, *B;                   // tensor cores: operand parts (dense_grad_sizes)
    uint32_t* error;
    uint32_t spin_limit;
};

struct NeuronArgs {
    const DevPop* pops;
    const int32_t* tile_pop;       // compaction tile -> population
    float *V, *m, *h, *n, *g0, *g1, *iext;
    float* isyn_rec;               // nullptr unless recording
    unsigned long long* ticket;    // monotone tile ticket: step epoch = ticket / num_tiles
    const unsigned long long* epoch_base;
    uint32_t* error;
    int32_t num_tiles;
    int32_t n_sub;
    float hs;                      // substep length dt / n_sub (ms)
    uint32_t spin_limit;
    uint32_t seed_lo, seed_hi;
};

struct PersistArgs {
    NeuronArgs n;
    const DevProj* projs;
    const int32_t* out_begin;      // [n_pops + 1] offsets into out_list
    const int32_t* out_list;       // projections grouped by pre population
    float* acc0;                   // [2][n_total] incoming events, channel 0
    float* acc1;                   // [2][n_total] incoming events, channel 1
    int32_t acc_stride;            // n_total
    int32_t n_steps;
    int32_t barrier_extra;         // test hook: arrivals the barrier waits for beyond the grid (0 normally)
    GridBarrier* bar;
};

struct PropArgs {
    const DevProj* projs;
    int32_t n_projs;
    int32_t chunk;                 // synapses per CSR work item
    const unsigned long long* ticket;   // the step delivered is epoch ticket / num_tiles - 1
    int32_t num_tiles;
};

// Memory obtained from the user allocator (or cudaMalloc).
struct Alloc {
    snn_allocator a{};
    bool have = false;
    void* stream = nullptr;
    void* get(size_t bytes);
    void put(void* p);
};

struct PopHost {
    snn_pop_desc d;
    int32_t offset, first_tile, n_tiles;
};

struct ProjHost {
    snn_proj_desc d;
    int64_t* csc_ptr = nullptr;    // graded: transposed copy
    int32_t* csc_pre = nullptr;
    uint16_t* csc_pre16 = nullptr;
    float* csc_w = nullptr;
    int64_t* csc_perm = nullptr;   // transposed position -> compressed-row position
    uint16_t* col16 = nullptr;     // graded: 16-bit post indices of the compressed rows (small post populations)
    float* dpart = nullptr;        // graded dense: partial rows of the forward product
    unsigned* dcount = nullptr;    // graded dense: per post block ticket
    int32_t dchunks = 1;           // graded dense: pre-row ranges of the forward product
    bool dstream = true;           // graded dense: stream W (evict-first) instead of keeping it in L2
    int64_t dld = 0;               // graded dense: row stride of dpart
    int64_t g_off = 0;
    float scale;
    int64_t nnz;
    int32_t max_row;
    int32_t mode = 0;          // 1: post-tiled bulk copies, 2: post-tiled segments
    int64_t* split = nullptr;
    int64_t* csplit = nullptr;     // cluster engine row segments
    int64_t* row_ptr = nullptr;
    int32_t* col = nullptr;
    float* w = nullptr;
};

}  // namespace snn

namespace snn {
// A dense projection shared by every instance of a batch (snn_add_shared_dense).
struct SharedDense {
    snn_dense_batch* h = nullptr;  // W, its BF16 parts and the spike matrix
    int32_t B = 0, n_pre = 0, n_post = 0, channel = 0;
    int32_t* pre_pop = nullptr;    // [B] population index of instance b's pre population (device)
    int32_t* pre_off = nullptr;    // [B] its SoA offset (device)
    int32_t* spk_off = nullptr;    // [B + 1] the step's spike lists (device), built each step
    int32_t* spk = nullptr;        // [B * n_pre]
    float* scale = nullptr;        // [B] s_b = gScale(nConn) * user_scale[b]
    float* G = nullptr;            // conductance channel of instance 0's post population
    int64_t ldg = 0;               // SoA distance between instances' post populations
    std::vector<int32_t> pre_pops; // host copy of pre_pop
};
}  // namespace snn

struct snn_net {
    snn::Alloc mem;
    std::vector<void*> owned;
    std::vector<snn::PopHost> pops;
    std::vector<snn::ProjHost> projs;
    double dt = 0.1;
    int32_t n_sub = 4;
    uint64_t seed = 0;
    uint32_t instance = 0;
    int32_t n_total = 0;           // padded SoA length
    int32_t num_tiles = 0;
    int sm_count = 148;
    int64_t l2_bytes = 0;
    // device state
    float *V = nullptr, *m = nullptr, *h = nullptr, *n = nullptr, *g0 = nullptr, *g1 = nullptr,
          *iext = nullptr, *isyn = nullptr;
    float* init_state = nullptr;   // 7 * n_total floats saved at creation
    int32_t* spk = nullptr;
    int32_t* nspk = nullptr;                  // [2 * n_pops]
    int32_t* nrn_count = nullptr;             // per-neuron spike counts (n_total)
    unsigned long long* d_events = nullptr;
    float* acc = nullptr;                     // persistent engine accumulators [2 channels][2 buffers][n_total]
    int32_t* out_begin = nullptr;
    int32_t* out_list = nullptr;
    snn::GridBarrier* bar = nullptr;
    int32_t engine = 2;                       // 0 plain, 1 persistent, 2 choose
    int32_t persist_steps = 1000;             // steps per persistent launch
    int32_t persist_grid = 0;                 // co-resident CTAs of the persistent kernel
    int32_t barrier_extra = 0;                // test hook of SNN_OPT_TEST_BARRIER_EXTRA
    int32_t cluster_size = 0, cluster_per_cta = 0;   // cluster engine plan (0: does not fit)
    int32_t cluster_seg_rows = 0;             // compressed rows whose CTA segments the cluster engine keeps in shared memory
    int32_t tiled = 2;                        // post-tiled rows: 0 off, 1 all compressed projections, 2 choose
    // graded (differentiable) networks
    bool graded = false;
    bool graded_narrow = false;               // 16-bit transposed pre indices
    int32_t graded_store = 1;                 // SNN_OPT_GRADED_STORE
    bool rec_stored = false;                  // the last recorded forward kept every step (traj_*)
    float* traj_state = nullptr;              // [T][5][n_total] step-start V, m, h, n, I_ext
    float* traj_r = nullptr;                  // [T][n_total] releases used by each step
    float* traj_G = nullptr;                  // [T][total_posts] G of each step
    size_t traj_cap_steps = 0;
    snn::GradProj* d_gprojs = nullptr;
    int32_t* in_begin = nullptr;
    int32_t* in_list = nullptr;
    int64_t total_posts = 0;
    int64_t spmv_items = 0;                   // work items of the graded forward product
    float *r = nullptr, *G = nullptr, *y = nullptr;
    double* d_grad_scale = nullptr;
    int64_t g_t = 0;                          // graded step counter
    // recorded forward
    int64_t rec_T = 0;
    int32_t rec_K = 0, rec_out_pop = -1, rec_n_out = 0;
    double rec_tau = 0.0;
    float* rec_ckpt = nullptr;                // [n_ckpt][6][n_total]
    size_t rec_ckpt_cap = 0;
    // segment buffers of the adjoint
    float *seg_state = nullptr, *seg_r = nullptr, *seg_G = nullptr;
    float *nu_step = nullptr, *nu_km = nullptr;
    float *adj = nullptr;                     // lV, lV_loc, lm, lh, ln (5 * n_total) + ly (n_total)
    int32_t seg_cap_K = 0;
    uint16_t *grad_A = nullptr, *grad_B = nullptr;   // operand parts of the dense weight gradient
    size_t grad_A_cap = 0, grad_B_cap = 0;
    int32_t dense_grad = 1;                   // dense weight gradient: 0 CUDA cores, 1 tensor cores
    std::vector<snn::SharedDense> shared;     // dense projections shared by all instances of a batch
    int32_t shared_engine = 2;                // their delivery: 0 CUDA cores, 1 tensor cores, 2 by spike density
    double shared_density = 0.03;             // spike density from which engine 2 uses the tensor cores
    unsigned long long* counters = nullptr;   // 2 * n_pops
    unsigned long long* ticket = nullptr;     // [0] ticket, [1] epoch base
    int32_t* tile_pop = nullptr;
    uint32_t* error = nullptr;
    snn::DevPop* d_pops = nullptr;
    snn::DevProj* d_projs = nullptr;          // one descriptor per projection
    snn::DevProj* d_dbg_proj = nullptr;       // one-projection scratch descriptor
    int32_t* d_dbg_spk = nullptr;
    int32_t dbg_cap = 0;
    bool dbg_staged = false;
    int32_t dbg_proj = 0;
    // options
    bool record_isyn = false;
    int64_t graph_steps = 100;
    int32_t prop_blocks = 0;
    int32_t chunk = 1024;
    uint32_t spin_limit = 1u << 22;
    // graph
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    int64_t graph_len = 0;
};

namespace snn {

// Thread-local error message helpers (api.cu).
snn_status fail(snn_status s, const std::string& msg);
snn_status cuda_fail(cudaError_t e, const char* what);

#define SNN_CK(call, what)                                       \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return snn::cuda_fail(e_, what);  \
    } while (0)

#define SNN_TRY(x)                    \
    do {                              \
        snn_status s_ = (x);          \
        if (s_ != SNN_OK) return s_;  \
    } while (0)

// Kernel launchers (neuron.cu, propagate.cu, csr.cu).
cudaError_t launch_neuron_step(const NeuronArgs& a, cudaStream_t s);
cudaError_t launch_init_state(const DevPop* pops, int n_pops_total, const int32_t* tile_pop,
                              int num_tiles, float* V, float* m, float* h, float* n, float* g0,
                              float* g1, float* iext, uint64_t seed, cudaStream_t s);
cudaError_t launch_propagate(const PropArgs& a, int blocks, cudaStream_t s);
int dense_rows_per_item();
int dense_posts_per_item();
cudaError_t launch_validate_csr(const int64_t* row_ptr, const int32_t* col, int32_t n_pre,
                                int32_t n_post, int64_t nnz, uint32_t* error, cudaStream_t s);
cudaError_t launch_densify(const int64_t* row_ptr, const int32_t* col, const float* w, int32_t n_pre,
                           int32_t n_post, float* W, cudaStream_t s);
cudaError_t launch_max_row(const int64_t* row_ptr, int32_t n_pre, int32_t* out, cudaStream_t s);
cudaError_t launch_event_list(const int64_t* row_ptr, const int32_t* col, const float* w,
                              const int32_t* spk, int32_t n, const int64_t* offsets,
                              int32_t* post_out, float* w_out, cudaStream_t s);
cudaError_t launch_row_lengths(const int64_t* row_ptr, const int32_t* spk, int32_t n,
                               int64_t* lens, cudaStream_t s);
cudaError_t launch_scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* scratch,
                            cudaStream_t s);
size_t scan_scratch_elems(int64_t n);
cudaError_t launch_csr_count(uint64_t seed, uint32_t tag, int64_t n_pre, int64_t n_post,
                             unsigned long long thr, int64_t* counts, cudaStream_t s);
cudaError_t launch_csr_fill(uint64_t seed, uint32_t tag, int64_t n_pre, int64_t n_post,
                            unsigned long long thr, const int64_t* row_ptr, int32_t* col,
                            cudaStream_t s);
cudaError_t launch_count_events(const DevProj* projs, int n_projs, unsigned long long* out, cudaStream_t s);
cudaError_t launch_row_splits(const int64_t* row_ptr, const int32_t* col, int32_t n_pre, int32_t n_tiles, int32_t P,
                              int64_t* split, cudaStream_t s);
cudaError_t propagate_occupancy(int* per_sm);   // resident row-kernel CTAs per SM (no dynamic smem)
cudaError_t launch_propagate_seg(const DevProj* q, const unsigned long long* ticket, int32_t num_tiles, int sm_count,
                                 cudaStream_t s);
cudaError_t launch_propagate_tiled(const DevProj* q, int32_t P, const unsigned long long* ticket, int32_t num_tiles,
                                   int sm_count, uint32_t* error, uint32_t spin_limit, cudaStream_t s);
constexpr int32_t kPostTile = 2048;          // posts per tile of the post-tiled propagation (8 KiB)
cudaError_t persistent_capacity(int sm_count, int* blocks);
// Compressed rows whose segment in a CTA's slice the cluster engine keeps in
// shared memory (16 bytes each).
constexpr int kClusterSegCacheRows = 2048;
// Dense delivery for batched instances that share W (dense_batch.cu): the
// spike-matrix capacity, and the launches without allocation (engine 0 CUDA
// cores, 1 tensor cores, 2 both gated on the device by spike count >= thr).
snn_status dense_batch_reserve(snn_dense_batch* h, int32_t B, cudaStream_t s);
cudaError_t dense_batch_launch(snn_dense_batch* h, int32_t B, const int32_t* spk_off, const int32_t* spk,
                               const float* scale, float* G, int64_t ldg, int32_t engine, int64_t thr, cudaStream_t s);
std::vector<int32_t> propagation_modes(const snn_net* net, int32_t tiled);
cudaError_t mark_state_live(snn_net* net, int32_t pop, bool g1, bool iext, cudaStream_t s);
int cluster_plan(int n_total, int n_pops, int n_projs, int* per_cta);
cudaError_t cluster_supported(int cl, int per_cta, int num_tiles, int seg_rows, bool* ok);
cudaError_t launch_cluster_splits(const int64_t* row_ptr, const int32_t* col, int32_t n_pre, int32_t post_soa,
                                  int32_t n_post, int32_t n_ranks, int32_t per_cta, int64_t* split, cudaStream_t s);
cudaError_t launch_cluster(const PersistArgs& a, int cl, int per_cta, int n_projs, int seg_rows, cudaStream_t s);
cudaError_t launch_graded_spmv(const GradedArgs& a, cudaStream_t s);
cudaError_t launch_graded_neuron(const GradedArgs& a, cudaStream_t s);
cudaError_t launch_graded_release_init(const GradedArgs& a, cudaStream_t s);
cudaError_t launch_graded_reverse(const GradedArgs& a, const AdjArgs& b, cudaStream_t s);
cudaError_t launch_graded_sddmm(const GradedArgs& a, const AdjArgs& b, int q, int64_t n_pre, float* grad_w, int L,
                                cudaStream_t s);
cudaError_t launch_scatter_csc(const float* w_csr, const int64_t* perm, float* w_csc, int64_t nnz, cudaStream_t s);
cudaError_t launch_finish_grad_scale(const double* acc, float* out, int n, cudaStream_t s);
int dense_fwd_chunks(int32_t n_pre, int32_t n_post, int sm_count);
cudaError_t launch_graded_dense_fwd(const float* W, const float* x, int32_t n_pre, int32_t n_post, float* Gq,
                                    float* part, int64_t ld_part, unsigned* count, int32_t chunks, bool stream,
                                    cudaStream_t s);
void dense_grad_sizes(int32_t n_pre, int32_t n_post, int32_t K, int64_t* mp, int64_t* np, int64_t* kp);
cudaError_t launch_dense_grad(const DenseGradArgs& g, cudaStream_t s);
cudaError_t launch_persistent(const PersistArgs& a, int grid, cudaStream_t s);
cudaError_t launch_set_epoch_base(unsigned long long* ticket, int num_tiles, cudaStream_t s);

unsigned long long bernoulli_threshold(double p);

// Device allocation owned by the network (released by snn_destroy).
template <typename T>
snn_status net_alloc(snn_net* net, T** out, size_t count, const char* what) {
    void* p = net->mem.get(count * sizeof(T));
    if (!p) return fail(SNN_ERR_OOM, std::string("device allocation failed: ") + what);
    net->owned.push_back(p);
    *out = static_cast<T*>(p);
    return SNN_OK;
}

// graded_api.cu
snn_status graded_setup(snn_net* net, cudaStream_t s);
snn_status graded_reset(snn_net* net, cudaStream_t s);
snn_status graded_step(snn_net* net, int64_t n_steps, cudaStream_t s);
bool graded_requested(const snn_proj_desc* projs, int n_projs);

}  // namespace snn
