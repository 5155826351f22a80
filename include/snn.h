/*
 * snn.h -- C-ABI of the GB300 spiking-network library.
 *
 * The library advances a conductance-based Hodgkin-Huxley network in time
 * steps of dt (Sec. 2 of Balaji, Yavuz, Nowotny, "Scalability and
 * optimization strategies for GPU enhanced neural networks"): every step
 * updates each neuron's membrane potential and Na/K gating variables, detects
 * threshold crossings into an ascending spike list, and delivers those spikes
 * over compressed-row connectivity (Sec. 3) whose conductances are scaled per
 * projection by gScale = k1 / (k2 + nConn) + k3 (Sec. 5.1, Tables 1 and 2).
 *
 * Conventions for every entry point:
 *   - Units: mV, ms, nS, pF, pA, Hz.
 *   - Pointers are plain host or device pointers; a flag next to each array
 *     says which.  The library never keeps a caller pointer past the call:
 *     inputs are deep-copied.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *     that only enqueue GPU work return before it finishes.
 *   - Every call returns an snn_status; SNN_OK is 0.  On any other value,
 *     snn_last_error() returns a message for the calling thread.  No C++
 *     exception crosses this boundary.
 *   - Ownership: an snn_net owns its device memory, obtained from the
 *     allocator given at creation (cudaMalloc when NULL) and released by
 *     snn_destroy.
 *   - Device-side failures (a bounded wait that ran out, a malformed input
 *     found on the GPU) set a sticky error word; the next call that
 *     synchronises (snn_read_state, snn_sync) returns it.
 */
#ifndef SNN_H
#define SNN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum snn_status {
    SNN_OK = 0,
    SNN_ERR_INVALID_ARG = 1, /* a size, index, flag or pointer is invalid */
    SNN_ERR_CSR = 2,         /* row starts not monotone, post index out of range or not ascending */
    SNN_ERR_GSCALE = 3,      /* nConn + k2 <= 0: the scaling law has no value (Sec. 5.1) */
    SNN_ERR_OOM = 4,         /* the allocator returned NULL */
    SNN_ERR_CUDA = 5,        /* a CUDA runtime call failed */
    SNN_ERR_TIMEOUT = 6,     /* a bounded device-side wait ran out */
    SNN_ERR_STATE = 7,       /* the call needs state the network does not have */
    SNN_ERR_SIZE = 8         /* a destination buffer is too small */
} snn_status;

enum { SNN_POP_HH = 0, SNN_POP_SOURCE = 1, SNN_POP_IZH = 2 };
enum { SNN_LAYOUT_CSR = 0, SNN_LAYOUT_DENSE = 1 };
enum { SNN_SYN_EXP = 0, SNN_SYN_GRADED = 1 };

/* State fields for snn_read_state / snn_write_state. */
enum {
    SNN_FIELD_V = 0,           /* float[n], membrane potential (mV) */
    SNN_FIELD_M = 1,           /* float[n], Na activation */
    SNN_FIELD_H = 2,           /* float[n], Na inactivation */
    SNN_FIELD_N = 3,           /* float[n], K activation */
    SNN_FIELD_G0 = 4,          /* float[n], conductance of channel 0 (nS) */
    SNN_FIELD_G1 = 5,          /* float[n], conductance of channel 1 (nS) */
    SNN_FIELD_IEXT = 6,        /* float[n], drive current (pA) */
    SNN_FIELD_ISYN = 7,        /* float[n], synaptic current of the last step (pA); needs SNN_OPT_RECORD_ISYN */
    SNN_FIELD_SPIKES = 8,      /* int32[nspk], spike list of the last step, handed out in ascending order (read only) */
    SNN_FIELD_NSPK = 9,        /* int32, length of that list (read only) */
    SNN_FIELD_SPIKE_COUNT = 10,/* int64, spikes since creation or reset (Fig. 1 avgSpike numerator) */
    SNN_FIELD_NAN_COUNT = 11,  /* int64, neuron-steps that ended with a NaN V (Fig. 1 sumNANs) */
    SNN_FIELD_NEURON_SPIKES = 12 /* int32[n], spikes of each neuron since creation or reset */
};

/* Options for snn_set_option. */
enum {
    SNN_OPT_RECORD_ISYN = 0,   /* 1: store I_syn of every step (for checking); default 0 */
    SNN_OPT_GRAPH_STEPS = 1,   /* steps per captured CUDA graph, 0 = no graph; default 100 */
    SNN_OPT_PROP_BLOCKS = 2,   /* CTAs of the propagation kernels; 0 = library choice */
    SNN_OPT_CHUNK = 3,         /* synapses per warp work item of the row kernel (multiple of 128) */
    SNN_OPT_SPIN_LIMIT = 4,    /* iterations of a bounded device wait before SNN_ERR_TIMEOUT */
    SNN_OPT_ENGINE = 5,        /* 0 plain (two kernels per step, graph replay), 1 persistent
                                  (one cooperative launch for many steps), 3 cluster (one
                                  thread-block cluster of up to 16 CTAs, events in distributed
                                  shared memory; networks up to 65,536 padded neurons),
                                  2 choose (default: cluster when the network fits one, else
                                  persistent when every tile gets its own resident CTA) */
    SNN_OPT_PERSIST_STEPS = 6, /* steps per persistent launch; default 1000 */
    SNN_OPT_TEST_BARRIER_EXTRA = 8, /* test hook, 0 (default) or 1: with 1 the persistent
                                  engine's grid barrier waits for one arrival that never
                                  comes, so every CTA runs out of SNN_OPT_SPIN_LIMIT and the
                                  next synchronising call returns SNN_ERR_TIMEOUT; snn_reset
                                  recovers the network */
    SNN_OPT_CLUSTER_CTAS = 9,  /* read only (snn_get_option): CTAs of the cluster engine's plan,
                                  0 when the network does not fit one cluster */
    SNN_OPT_SHARED_DENSE = 11, /* delivery of dense projections shared by a batch's instances
                                  (snn_add_shared_dense): 0 CUDA cores, 1 tensor cores, 2 chosen
                                  on the device each step (default: tensor cores when at least
                                  3 % of the pre neurons of all instances spiked) */
    SNN_OPT_GRADED_STORE = 12, /* snn_forward_record of a graded network: 1 (default) keeps every
                                  step's start state, releases and G on the device when they take
                                  at most a quarter of the free device memory, so that
                                  snn_backward reads them instead of recomputing each checkpoint
                                  segment (same results, bit for bit); 0 always recomputes */
    SNN_OPT_DENSE_GRAD = 10,   /* weight gradient of dense graded projections in snn_backward:
                                  0 CUDA cores (FP32 products), 1 tensor cores (default; three
                                  BF16 parts of each operand, six products, FP32 accumulation) */
    SNN_OPT_TILED = 7          /* compressed-row propagation of the plain engine: 0 one warp per
                                  row chunk with global atomics, 1 post-tiled through shared
                                  memory by bulk copies, 2 choose (default), 3 post-tiled
                                  segments streamed by warps into shared memory */
};

/* A population.  kind SNN_POP_HH: Traub-Miles HH neurons with the given
 * conductances; kind SNN_POP_SOURCE: Poisson spike sources at src_rate_hz;
 * kind SNN_POP_IZH: the cortical neurons of the paper's first network (Sec.
 * 5.1, its ref. [9]): v' = 0.04 v^2 + 5 v + 140 - u + I, u' = a (b v - u),
 * spike and reset v <- c, u <- u + d when v >= v_thresh; v takes n_substeps
 * Euler substeps per dt, u one step of dt with the new v.  Per neuron one
 * uniform r (drawn from the seed) gives a = izh[0] + izh[1] r,
 * b = izh[2] + izh[3] r, c = izh[4] + izh[5] r^2, d = izh[6] + izh[7] r^2.
 * I = bias + noise_sigma * z + g0 + g1: z is the per-step Irwin-Hall normal
 * draw (12 uniforms of 20 bits from the seed, minus 6), and the synaptic
 * input is the current g0 + g1 (E_syn unused; tau_syn 0 makes every event a
 * one-step pulse).  u starts at b v0; v0 as for HH. */
typedef struct snn_pop_desc {
    int32_t kind;
    int32_t n;                 /* neurons, 0 <= n < 2^30 */
    double C, gNa, ENa, gK, EK, gL, EL;  /* pF, nS, mV (HH only) */
    double E_syn[2];           /* reversal potential of conductance channel 0 / 1 (mV) */
    double tau_syn[2];         /* decay time constant of channel 0 / 1 (ms); <= 0 clears each step */
    double v_thresh;           /* spike threshold (mV): V(t) < v_thresh <= V(t+dt) */
    double src_rate_hz;        /* SNN_POP_SOURCE rate */
    double drive_rate_hz;      /* HH: Bernoulli(rate*dt) drive events per step; 0 = no drive */
    double drive_amp;          /* pA added to I_ext by each drive event */
    double drive_tau;          /* ms, decay of I_ext */
    const float* v0;           /* n initial potentials; NULL = EL.  Gating starts at steady state. */
    int32_t v0_on_device;      /* 1 if v0 is a device pointer */
    int32_t reserved;
    double izh[8];             /* SNN_POP_IZH: a0, a1, b0, b1, c0, c2, d0, d2 (see above) */
    double noise_sigma;        /* SNN_POP_IZH: standard deviation of the per-step input current */
    double bias;               /* SNN_POP_IZH: constant input current */
} snn_pop_desc;

/* A projection from population `pre` to `post`.  Input connectivity is either
 * compressed rows (Sec. 3: row_ptr[n_pre+1] int64, col[nnz] int32 post
 * indices ascending within each row, w[nnz] float weights in nS) or, with
 * input_dense = 1, a row-major n_pre x n_post weight matrix in w.  `layout`
 * is the storage the library keeps and propagates from (Eq. 1 vs Eq. 2).
 * Conductance scale s = (k1 / (k2 + nConn) + k3) * user_scale, computed in
 * FP64 and rounded to FP32; nConn = n_conn if > 0, else density * n_pre. */
typedef struct snn_proj_desc {
    int32_t pre, post;
    int32_t layout;            /* SNN_LAYOUT_CSR or SNN_LAYOUT_DENSE */
    int32_t channel;           /* post conductance channel 0 or 1 */
    int32_t synapse;           /* SNN_SYN_EXP (spiking) or SNN_SYN_GRADED */
    int32_t on_device;         /* 1 if row_ptr, col, w are device pointers */
    int32_t input_dense;       /* 1 if w is a dense n_pre x n_post matrix */
    int32_t reserved;
    int64_t nnz;
    const int64_t* row_ptr;
    const int32_t* col;
    const float* w;
    double k1, k2, k3;         /* scaling law constants */
    double density;            /* p */
    double n_conn;             /* explicit nConn, or <= 0 to use density * n_pre */
    double user_scale;         /* extra factor c */
    double v_thr, v_slope;     /* graded release 1 / (1 + exp((v_thr - V_pre) / v_slope)) */
} snn_proj_desc;

/* Device memory provider.  alloc returns a device pointer of at least
 * `bytes` (aligned to 256 B) usable on `stream`, or NULL; free releases it. */
typedef struct snn_allocator {
    void* (*alloc)(size_t bytes, void* stream, void* ctx);
    void (*free)(void* ptr, void* stream, void* ctx);
    void* ctx;
} snn_allocator;

typedef struct snn_net snn_net;

/* Creates a network (Sec. 2 model, Sec. 3 storage, Sec. 5.1 scaling).
 * Copies every input array, validates connectivity on the GPU
 * (SNN_ERR_CSR), computes each projection's scale (SNN_ERR_GSCALE at the
 * law's pole), initialises V from v0 and m, h, n at their steady state, and
 * zeroes conductances, drive currents and counters.  Synchronises `stream`.
 * `rng_instance` (< 2^24) is folded into every random-number counter so that
 * instance b of a batch reproduces a stand-alone network created with b.
 * At most 4096 populations and 4096 projections. */
snn_status snn_create_network(const snn_pop_desc* pops, int32_t n_pops,
                              const snn_proj_desc* projs, int32_t n_projs,
                              double dt, int32_t n_substeps, uint64_t seed, uint32_t rng_instance,
                              const snn_allocator* alloc, void* stream, snn_net** out);

/* One network instance of a batch. */
typedef struct snn_net_desc {
    const snn_pop_desc* pops;
    int32_t n_pops;
    const snn_proj_desc* projs;
    int32_t n_projs;
    uint32_t rng_instance;     /* folded into the instance's random-number counters (< 2^24) */
    int32_t reserved;
} snn_net_desc;

/* Creates one network object that holds n_instances independent networks of
 * any sizes (the batched form: many instances with their own conductance
 * scale factors, as in the paper's sweep over scaling factors, Sec. 2 and
 * Fig. 1).  Their populations and projections are packed one after another:
 * instance b's population k becomes population (sum of n_pops of instances
 * < b) + k of the batch, and likewise for projections, so every other call
 * (snn_step, snn_read_state, counters) addresses them by those indices.  No
 * projection crosses instances.  Each instance draws the same random numbers
 * as a stand-alone network created with its rng_instance.  Up to 4096
 * populations and 4096 projections in total; errors as snn_create_network. */
snn_status snn_create_batch(const snn_net_desc* nets, int32_t n_instances, double dt, int32_t n_substeps,
                            uint64_t seed, const snn_allocator* alloc, void* stream, snn_net** out);

/* Adds a dense projection (Eq. 2 storage) that every instance of a batch
 * shares: instance b's population first_post + b * pops_per_instance
 * receives, on conductance channel `channel`, s_b * W[i][j] for each spike i
 * of its population first_pre + b * pops_per_instance, with one step of
 * delay like every projection.  W is n_pre x n_post row-major FP32 (host or
 * device, copied; n_pre / n_post the populations' sizes, the same in every
 * instance), s_b = (k1 / (k2 + nConn) + k3) * user_scale[b] (Sec. 5.1; nConn
 * = n_conn if > 0, else density * n_pre; user_scale: host, n_instances
 * doubles).  Each step delivers all instances at once, as the product of the
 * step's 0/1 spike matrix (instances x n_pre) with W: on the tensor cores
 * (W split into three BF16 parts, FP32 accumulation, as snn_dense_batch) or
 * on the CUDA cores, see SNN_OPT_SHARED_DENSE.  The instances' post
 * populations must lie evenly spaced in the batch (instances of identical
 * shape): SNN_ERR_INVALID_ARG otherwise; SNN_ERR_GSCALE for nConn + k2 <= 0.
 * A network with shared projections steps in the plain engine.  Synchronises
 * `stream`. */
snn_status snn_add_shared_dense(snn_net* net, int32_t first_pre, int32_t first_post, int32_t pops_per_instance,
                                int32_t n_instances, const float* w, int32_t w_on_device, int32_t channel, double k1,
                                double k2, double k3, double density, double n_conn, const double* user_scale,
                                void* stream);

/* Releases the network and all its device memory (synchronises its streams). */
snn_status snn_destroy(snn_net* net);

/* Enqueues n_steps time steps on `stream`.  Each step: Poisson sources draw
 * spikes; driven neurons draw drive events; I_syn = sum_c g_c (E_c - V);
 * n_substeps forward-Euler substeps of V, m, h, n; upward threshold crossings
 * are listed in ascending order; conductances and drive decay by
 * exp(-dt / tau); each spike adds s * w to its targets' conductance (one-step
 * delay).  Full blocks of SNN_OPT_GRAPH_STEPS steps replay a captured graph.
 * Does not synchronise; returns a sticky device error seen earlier. */
snn_status snn_step(snn_net* net, int64_t n_steps, void* stream);

/* Waits for `stream` and returns any sticky device error (SNN_ERR_TIMEOUT,
 * SNN_ERR_CSR). */
snn_status snn_sync(snn_net* net, void* stream);

/* Copies a state field of population `pop` into dst (host or device).
 * `bytes` must cover the field (SNN_ERR_SIZE otherwise); for SNN_FIELD_SPIKES
 * it must cover n * 4 bytes.  Synchronises `stream`. */
snn_status snn_read_state(snn_net* net, int32_t pop, int32_t field, void* dst, size_t bytes,
                          int32_t dst_is_device, void* stream);

/* Overwrites a float state field (V, M, H, N, G0, G1, IEXT) of population
 * `pop` from src (host or device), `bytes` = n * 4.  Synchronises `stream`. */
snn_status snn_write_state(snn_net* net, int32_t pop, int32_t field, const void* src, size_t bytes,
                           int32_t src_is_device, void* stream);

/* Restores the state the network had at creation, sets the step counter
 * (and hence the random-number counters) back to 0 and clears a sticky
 * device error.  Enqueued on `stream`. */
snn_status snn_reset(snn_net* net, void* stream);

/* Sets an SNN_OPT_* option (see the enum). */
snn_status snn_set_option(snn_net* net, int32_t option, int64_t value);

/* Reads the current value of an SNN_OPT_* option into *value (host
 * pointer).  SNN_ERR_INVALID_ARG for an unknown option or a NULL pointer. */
snn_status snn_get_option(const snn_net* net, int32_t option, int64_t* value);

/* Engine snn_step uses with the current options: 0 plain, 1 persistent, 3 cluster. */
snn_status snn_get_engine(snn_net* net, int32_t* engine);

/* Steps simulated since creation or the last reset (synchronises `stream`). */
snn_status snn_get_step(snn_net* net, int64_t* step, void* stream);

/* Synaptic events delivered since creation or reset: the sum over projections
 * and spikes of the spiking pre neuron's row length (n_post for dense
 * storage), from the per-neuron spike counts.  Synchronises `stream`. */
snn_status snn_synaptic_events(snn_net* net, int64_t* events, void* stream);

/* Launches one phase of a step exactly as snn_step does, for timing single
 * kernels: phase 0 = neuron update with spike compaction, 1 = propagation,
 * 2 = one persistent launch of SNN_OPT_PERSIST_STEPS complete steps,
 * 3 = the propagation kernel again on the list last staged by
 * snn_debug_propagate (SNN_ERR_STATE if none), 4 = one cluster launch of
 * SNN_OPT_PERSIST_STEPS complete steps (SNN_ERR_STATE if it does not fit).
 * A neuron phase without its propagation advances the state without
 * delivering spikes.  Enqueued on `stream`. */
snn_status snn_launch_phase(snn_net* net, int32_t phase, void* stream);

/* Conductance scale s of projection `proj` as the GPU uses it (FP32). */
snn_status snn_proj_scale(snn_net* net, int32_t proj, float* scale);

/* Number of synapses stored for projection `proj` (nnz; n_pre * n_post for dense). */
snn_status snn_proj_nnz(snn_net* net, int32_t proj, int64_t* nnz);

/* Which kernel delivers the spikes of projection `proj` in the plain engine
 * (Sec. 3's compressed-row propagation and its post-tiled forms), as chosen
 * by SNN_OPT_TILED: *mode = 0 one warp per row chunk (k_propagate; also every
 * dense projection), 1 one bulk-copied piece per row and post tile
 * (k_propagate_tiled), 2 the rows' tile segments streamed by warps into a
 * shared accumulator (k_propagate_seg).  SNN_ERR_INVALID_ARG for a bad projection or
 * a NULL `mode`. */
snn_status snn_proj_mode(snn_net* net, int32_t proj, int32_t* mode);

/* Runs the production propagation kernel of projection `proj` once on the
 * given ascending spike list of its pre population (host or device, n
 * entries), adding s * w to the post conductances.  For checking delivery
 * against the dense product of Sec. 3's Eq. 2 storage.  Synchronises. */
snn_status snn_debug_propagate(snn_net* net, int32_t proj, const int32_t* spk, int32_t n,
                               int32_t spk_on_device, void* stream);

/* Event list of a spike list over projection `proj` (compressed rows only):
 * for each spike in list order, the (post index, weight) pairs of its row in
 * storage order, written to device arrays post_out / w_out of `capacity`
 * entries.  *n_events receives the total; SNN_ERR_SIZE if it exceeds
 * capacity (nothing written).  Spikes are host or device.  Synchronises. */
snn_status snn_event_list(snn_net* net, int32_t proj, const int32_t* spk, int32_t n,
                          int32_t spk_on_device, int32_t* post_out, float* w_out,
                          int64_t capacity, int64_t* n_events, void* stream);

/* Compressed-row connectivity drawn on the GPU from a seed (Sec. 3 format):
 * one Bernoulli(p) draw per (pre i, post j) pair, event when word (j mod 4)
 * of Philox4x32-10(counter = (j / 4, i, tag, 3), key = seed) is below
 * round(p * 2^32).  Pass 1 writes row_ptr[n_pre + 1] (device) and *nnz
 * (host); pass 2 writes col[nnz] (device), ascending within each row.
 * Scratch memory comes from `alloc` (cudaMalloc when NULL).  Synchronises
 * `stream`.  n_pre, n_post < 2^31; 0 <= p <= 1. */
snn_status snn_csr_bernoulli_rows(uint64_t seed, uint32_t tag, int64_t n_pre, int64_t n_post,
                                  double p, int64_t* row_ptr, int64_t* nnz,
                                  const snn_allocator* alloc, void* stream);
snn_status snn_csr_bernoulli_fill(uint64_t seed, uint32_t tag, int64_t n_pre, int64_t n_post,
                                  double p, const int64_t* row_ptr, int32_t* col, void* stream);

/* Largest n_pre accepted by snn_csr_bernoulli_rows_noalloc. */
#define SNN_NOALLOC_MAX_ROWS 16777216

/* Same result as snn_csr_bernoulli_rows (bit for bit), without allocating.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory when they build connectivity -- code whose
 * device memory all belongs to a pool or budget it must stay inside, and
 * loops that must not call cudaMalloc / cudaFree at all (cudaFree may wait
 * for the whole device; this call waits on `stream` only).
 * Row counts are written into row_ptr itself; the only scratch is a fixed
 * array of SNN_NOALLOC_MAX_ROWS / 1024 + 1 int64 (128 KiB) in device memory,
 * held by every GPU that loads the library until the process exits.
 * The first call on a device does the set-up: with the device current it
 * looks up that array's device address, which later calls reuse; make that
 * first call before any stream capture.  The address is kept per device
 * context, so the first call after cudaDeviceReset looks it up again.
 * Every call on a device shares the array: calls whose GPU work overlaps
 * (different streams, no ordering between them) race and give wrong rows;
 * calls ordered on one stream are safe.  Each call writes every scratch entry
 * it reads, so nothing needs clearing between calls.
 * n_pre > SNN_NOALLOC_MAX_ROWS returns SNN_ERR_SIZE before any GPU work.
 * Calls no cudaMalloc, cudaFree or allocating library routine.
 * Synchronises `stream`; *nnz (host) receives row_ptr[n_pre]. */
snn_status snn_csr_bernoulli_rows_noalloc(uint64_t seed, uint32_t tag, int64_t n_pre, int64_t n_post,
                                          double p, int64_t* row_ptr, int64_t* nnz, void* stream);

/* ---- dense delivery for batched instances, on the tensor cores ------------ */
/* Many network instances that share one dense projection W (Eq. 2 storage)
 * receive, per step, G[b][j] += s_b * sum over the spikes i of instance b of
 * W[i][j].  On the tensor cores that is one product of the spike matrix S
 * (B x n_pre, 0/1, exact in BF16) with W, which is split once into three BF16
 * parts W = hi + mid + lo (each the BF16 rounding of what the previous parts
 * left, together W's 24 significant bits); the three products accumulate in
 * FP32 in tensor memory (tcgen05), so the result has FP32-sum accuracy. */
typedef struct snn_dense_batch snn_dense_batch;

/* Copies W (n_pre x n_post row-major FP32, host or device) and prepares its
 * parts.  Device memory through `alloc` (may be NULL: cudaMalloc).
 * SNN_ERR_INVALID_ARG for sizes < 1 or n_pre * n_post > 2^31.  Synchronises
 * `stream`. */
snn_status snn_dense_batch_create(const float* W, int32_t n_pre, int32_t n_post, int32_t w_on_device,
                                  const snn_allocator* alloc, void* stream, snn_dense_batch** out);

/* Frees the handle and its device memory (synchronises the device). */
snn_status snn_dense_batch_destroy(snn_dense_batch* h);

/* Delivers one step for B instances; all pointers are device pointers:
 * spk_off[B + 1] int32 offsets into spk (pre indices of each instance's
 * spikes), scale[B], G rows of n_post floats with a stride of ldg floats
 * (ldg >= n_post), accumulated.  engine 0: CUDA cores (each thread sums its
 * four posts over the instance's spike rows); engine 1: tensor cores (S is
 * built in device scratch owned by the handle, then one 128 x 128 output
 * tile per CTA).  Enqueued on `stream`; errors of the kernels (a spike index
 * outside [0, n_pre), a bounded wait that ran out) are reported by
 * snn_dense_batch_check. */
snn_status snn_dense_batch_deliver(snn_dense_batch* h, int32_t B, const int32_t* spk_off, const int32_t* spk,
                                   const float* scale, float* G, int64_t ldg, int32_t engine, void* stream);

/* Synchronises `stream` and reports a sticky kernel error of the handle:
 * SNN_ERR_INVALID_ARG (spike index out of range) or SNN_ERR_TIMEOUT. */
snn_status snn_dense_batch_check(snn_dense_batch* h, void* stream);

/* ---- weight gradient of a dense projection: rank-K update ---------------- */
/* D[i][j] += sum over t < K of R[t][i] N[j][t] (i < m, j < n): the adjoint
 * weight gradient of a dense graded projection (Eq. 2 storage) over one
 * checkpoint segment of K steps, with R the segment's releases of the pre
 * population (step-major) and N the segment's dL/dG of the posts
 * (time-contiguous per post); snn_backward runs it for every dense
 * projection.  On the tensor cores both operands are split into three BF16
 * parts and the six products whose weight reaches 2^-24 of the result
 * accumulate in FP32 in tensor memory (tcgen05), so D receives an FP32-
 * accurate sum; the CUDA-core engine forms FP32 products directly. */
typedef struct snn_dense_grad snn_dense_grad;

/* A handle owning the operand-part scratch (grown on demand) and an error
 * word; device memory through `alloc` (may be NULL: cudaMalloc). */
snn_status snn_dense_grad_create(const snn_allocator* alloc, void* stream, snn_dense_grad** out);

/* Frees the handle and its device memory (synchronises the device). */
snn_status snn_dense_grad_destroy(snn_dense_grad* h);

/* Enqueues one update on `stream`.  Device pointers: R[t * ldr + i]
 * (ldr >= m), N[j * ldn + t] (ldn >= K), D[i * ldd + j] (ldd >= n),
 * accumulated.  engine 0: CUDA cores, 1: tensor cores.  m, n >= 0,
 * 0 <= K <= 512; SNN_ERR_INVALID_ARG otherwise.  A bounded wait that ran out
 * is reported by snn_dense_grad_check. */
snn_status snn_dense_grad_run(snn_dense_grad* h, const float* R, int64_t ldr, const float* N, int64_t ldn,
                              int32_t m, int32_t n, int32_t K, float* D, int64_t ldd, int32_t engine, void* stream);

/* Synchronises `stream` and reports a sticky kernel error of the handle
 * (SNN_ERR_TIMEOUT). */
snn_status snn_dense_grad_check(snn_dense_grad* h, void* stream);

/* ---- parameters ----------------------------------------------------------- */
/* Replaces the conductance scale s of projection `proj` (rounded to FP32). */
snn_status snn_set_scale(snn_net* net, int32_t proj, double scale);

/* Replaces the weights of projection `proj`, host or device: the nnz weights
 * (nS) in compressed-row order, or for dense storage the n_pre x n_post
 * matrix in row-major order.  Synchronises `stream`. */
snn_status snn_set_weights(snn_net* net, int32_t proj, const float* w, int32_t on_device, void* stream);

/* ---- differentiable form (graded synapses) ---------------------------------
 * A network whose projections all have synapse = SNN_SYN_GRADED uses graded
 * release r = 1 / (1 + exp((v_thr - V_pre) / v_slope)) instead of spikes:
 * each step, G_q[k] = sum_i w_ik r_i and I_syn_k = sum_q s_q (E_q - V_k) G_q[k]
 * (E_q: the post population's reversal potential of the projection's
 * channel), then the Euler substeps; spike counts are still kept.  The paper
 * fixes no synapse model (Sec. 2); this graded one makes the output y below a
 * smooth function of the scales s_q (Sec. 5.1) and the weights.  Graded
 * projections use compressed rows or dense storage (Eq. 2, every pair a
 * weight); populations must be HH. */

/* Runs n_steps steps from the creation state (it resets the network first)
 * and writes the output filter: y_out[t][k] = y_k(t + 1) (device, n_steps x
 * n_out floats, step-major, owned by the caller), where y follows the output
 * population's V with y += (dt / tau_f)(V - y), starting at V(0).  Any loss
 * L(y) is the caller's; snn_backward takes its gradient dL/dy.  Keeps, for
 * snn_backward, every step's start state, releases and G when they fit
 * (SNN_OPT_GRADED_STORE), else the state every checkpoint_every steps
 * (1..512); checkpoint_every is also the adjoint's segment length.
 * Synchronises `stream`.  SNN_ERR_STATE for a spiking network;
 * SNN_ERR_INVALID_ARG for y_out == NULL or bad sizes. */
snn_status snn_forward_record(snn_net* net, int64_t n_steps, int32_t checkpoint_every, int32_t out_pop,
                              double tau_f, float* y_out, void* stream);

/* Gradient of a loss L(y) of the last recorded forward's y with respect to
 * every projection's scale (grad_scale: device, n_projs floats) and weights
 * (grad_w: host array of n_projs device pointers, each nnz floats in
 * compressed-row order, or n_pre x n_post row-major for dense storage),
 * given dL_dy (device, n_steps x n_out floats in y_out's layout, read during
 * the call, owned by the caller), by the discrete adjoint of the recorded
 * steps: each segment's states are read from the kept trajectory or
 * recomputed from its checkpoint (the same bits), then swept in reverse
 * (filter, substeps, synaptic current, pre-synaptic gather), and the weight
 * gradients of the segment are summed over its steps in one pass (for dense
 * storage a rank-K update, see snn_dense_grad_run and SNN_OPT_DENSE_GRAD).
 * Overwrites the outputs.  SNN_ERR_STATE without a recorded forward.
 * Synchronises `stream`. */
snn_status snn_backward(snn_net* net, const float* dL_dy, float* grad_scale, float* const* grad_w, void* stream);

/* Enqueues the graded forward product alone (Sec. 2's synaptic input of the
 * graded form, G_q[j] = sum_i w_ij r_i over the compressed-row projections,
 * from the current releases, into the network's G vector), for timing the
 * kernel: the state does not advance.  SNN_ERR_STATE for a spiking
 * network. */
snn_status snn_graded_launch_product(snn_net* net, void* stream);

/* ---- checkpoint / resume --------------------------------------------------
 * A snapshot holds the whole dynamic state: V, m, h, n, conductances, drive
 * currents, spike lists and lengths, all counters, the persistent engine's
 * accumulators and the step counter (so random numbers continue where they
 * left off).  Loading it into the same network (or one created from the same
 * description) and stepping reproduces the uninterrupted run up to the order
 * of floating-point atomic adds.  Buffers are host or device; the caller
 * owns them.  snn_save_state synchronises `stream` and returns a sticky error
 * first; snn_load_state returns SNN_ERR_STATE for a snapshot of another shape
 * and SNN_ERR_SIZE for a short buffer. */
snn_status snn_state_size(snn_net* net, size_t* bytes);
snn_status snn_save_state(snn_net* net, void* dst, size_t bytes, int32_t dst_is_device, void* stream);
snn_status snn_load_state(snn_net* net, const void* src, size_t bytes, int32_t src_is_device, void* stream);

/* ---- autotuning ----------------------------------------------------------- */
typedef struct snn_tuning {
    int32_t engine;            /* SNN_OPT_ENGINE chosen (0 plain, 1 persistent) */
    int32_t prop_blocks;       /* SNN_OPT_PROP_BLOCKS */
    int32_t chunk;             /* SNN_OPT_CHUNK */
    int32_t tiled;             /* SNN_OPT_TILED */
    double us_per_step;        /* trial time of the chosen configuration */
    int32_t cached;            /* 1 if taken from the in-process cache */
    int32_t reserved;
} snn_tuning;

/* Times candidate launch configurations (engine, propagation CTAs, row chunk,
 * post-tiled rows) on trial runs of `trial_steps` steps started from a
 * snapshot of the current state, applies the fastest, and restores the
 * snapshot so the simulation continues unchanged.  Results are cached per
 * device and network shape for the life of the process.  `result` may be
 * NULL.  Synchronises `stream`.  The paper's own block-size rule is
 * occupancy-based (Sec. 3); this replaces it with measurement. */
snn_status snn_autotune(snn_net* net, int32_t trial_steps, snn_tuning* result, void* stream);

/* Applies the configuration of the paper's occupancy rule (Sec. 3: the block
 * and grid sizes follow from the resident warps per SM, not from a
 * measurement): the plain two-kernel step, propagation grid = SMs x resident
 * row-kernel CTAs per SM, row chunk 1024, no post tiling.  It times that
 * configuration with the same trial procedure as snn_autotune (state restored
 * afterwards) and reports it in `result` (may be NULL; `cached` is 0), so the
 * tuned-versus-occupancy speed-up can be read off.  SNN_ERR_STATE for a
 * graded network.  Synchronises `stream`. */
snn_status snn_occupancy_config(snn_net* net, int32_t trial_steps, snn_tuning* result, void* stream);

/* Message of the last failed call on this thread ("" if none). */
const char* snn_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SNN_H */
