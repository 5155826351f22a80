/*
 * FP64 CPU oracle for one time step of a conductance-based Hodgkin-Huxley
 * spiking network with connection-density-dependent conductance scaling.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file; only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no source with the CUDA library.
 *
 * What the paper fixes and what this file follows:
 *   - Sec. 2: HH neurons advanced at discretised time steps; synaptic
 *     conductance scaled per projection; NaN states counted.
 *   - Sec. 3: compressed-row synapse storage (values, post indices and a
 *     per-pre row start array) and the memory formulas Eq. 1 / Eq. 2.
 *   - Sec. 5.1: gScale = k1 / (k2 + nConn) + k3 (also written as
 *     (gScale - k3)(nConn + k2) = k1), with Table 1 / Table 2 constants;
 *     Fig. 1 defines the per-run average spike count and NaN count.
 * What the paper leaves open and the reading taken here (each one is also
 * listed with the design notes of the repository):
 *   - HH model: Traub-Miles rates (V in mV, rates in 1/ms), units nS, pF,
 *     pA, mV, ms.  Linoid rates evaluated as k * x / expm1(x).
 *   - Integrator: forward Euler with n_sub substeps per step; the synaptic
 *     current is computed once from step-start V and held; every right-hand
 *     side is evaluated at the substep start.
 *   - Spike: upward crossing of v_thresh between step-start and step-end V.
 *   - Synapse: exponential conductance, jump s*w per event, decay
 *     exp(-dt/tau) applied before the step's events are added (one step of
 *     transmission delay).  Two conductance channels per neuron.
 *   - Random numbers: Philox4x32-10, compared as integers against
 *     round(p * 2^32), so CPU and GPU draw identical bits.
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,       */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11).  Each round      */
/* multiplies words 0 and 2 by fixed odd constants, swaps halves and xors  */
/* in the key; the key advances by the Weyl constants between rounds.      */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c[0];
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c[3] ^ k1;
        uint32_t n3 = lo0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* Stream identifiers carried in counter word 3. */
enum { STREAM_SOURCE = 1, STREAM_DRIVE = 2, STREAM_CSR = 3, STREAM_IZH_PARAM = 5, STREAM_IZH_NOISE = 6 };

/* One 32-bit draw: key = seed, counter = (a, b, tag, stream), word `word`. */
static uint32_t draw_u32(uint64_t seed, uint32_t a, uint32_t b, uint32_t tag,
                         uint32_t stream, int word)
{
    uint32_t ctr[4] = {a, b, tag, stream};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t out[4];
    oracle_philox4x32_10(ctr, key, out);
    return out[word];
}

/* Per-neuron parameter draw r of an Izhikevich population: the top 24 bits
 * of word 0 of Philox(counter = (i, 0, tag, STREAM_IZH_PARAM)) times 2^-24,
 * uniform on [0, 1) and exact in FP32 and FP64. */
double oracle_izh_r(uint64_t seed, uint32_t tag, uint32_t i)
{
    return (double)(draw_u32(seed, i, 0, tag, STREAM_IZH_PARAM, 0) >> 8) * 0x1p-24;
}

/* Approximately normal input noise of neuron i at step t (Irwin-Hall: the
 * sum of 12 uniforms minus 6 has mean 0 and variance 1): the top 20 bits of
 * the 12 words of Philox(counter = (i, t, tag, STREAM_IZH_NOISE + k)),
 * k = 0, 1, 2, summed as integers S < 12 * 2^20, z = (S - 6 * 2^20) 2^-20.
 * z is exact in FP32, so both sides draw identical values. */
double oracle_izh_noise(uint64_t seed, uint32_t tag, uint32_t t, uint32_t i)
{
    int64_t S = 0;
    for (uint32_t k = 0; k < 3; ++k) {
        uint32_t ctr[4] = {i, t, tag, STREAM_IZH_NOISE + k};
        uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
        uint32_t out[4];
        oracle_philox4x32_10(ctr, key, out);
        for (int w = 0; w < 4; ++w) S += out[w] >> 12;
    }
    return (double)(S - 6 * (1 << 20)) * 0x1p-20;
}

/* Integer Bernoulli threshold round(p * 2^32), clamped to [0, 2^32]; an
 * event happens when the 32-bit draw is strictly below it. */
uint64_t oracle_bernoulli_threshold(double p)
{
    if (!(p > 0.0)) return 0;
    double t = nearbyint(p * 4294967296.0);
    if (t >= 4294967296.0) return 4294967296ull;
    return (uint64_t)t;
}

/* ------------------------------------------------------------------------ */
/* Conductance scaling law, Sec. 5.1 (Tables 1 and 2 give k1, k2, k3).      */
/* Returns 0 and writes gScale, or -1 when nConn + k2 <= 0 (the hyperbola's */
/* pole, where the law is undefined).                                       */
/* ------------------------------------------------------------------------ */
int oracle_gscale(double k1, double k2, double k3, double n_conn, double* out)
{
    double den = k2 + n_conn;
    if (!(den > 0.0)) return -1;
    *out = k1 / den + k3;
    return 0;
}

/* Memory words of Sec. 3: Eq. 2 (dense) is nPre * nPost.  Eq. 1 (sparse) as
 * printed adds nPostSynN, but the text says the row-start array has one
 * entry per pre-synaptic neuron; the reading taken is 2*nNZ values+indices,
 * nPre + 1 row starts (the extra one closes the last row) and 1 word for the
 * stored nNZ integer. */
int64_t oracle_memory_words(int64_t nnz, int64_t n_pre, int64_t n_post, int dense)
{
    if (dense) return n_pre * n_post;
    return 2 * nnz + (n_pre + 1) + 1;
}

/* ------------------------------------------------------------------------ */
/* Traub-Miles rate functions (1/ms) with V in mV.                          */
/* ------------------------------------------------------------------------ */
static double xm1(double x)   /* x / (exp(x) - 1), continuous at x = 0 */
{
    if (fabs(x) < 1e-6) return 1.0 - 0.5 * x + x * x / 12.0;
    return x / expm1(x);
}

void oracle_hh_rates(double V, double out[6])
{
    /* alpha_m = 0.32 (-52 - V) / (exp((-52 - V)/4) - 1) */
    out[0] = 0.32 * 4.0 * xm1((-52.0 - V) / 4.0);
    /* beta_m  = 0.28 (V + 25) / (exp((V + 25)/5) - 1) */
    out[1] = 0.28 * 5.0 * xm1((V + 25.0) / 5.0);
    /* alpha_h = 0.128 exp((-48 - V)/18) */
    out[2] = 0.128 * exp((-48.0 - V) / 18.0);
    /* beta_h  = 4 / (exp((-25 - V)/5) + 1) */
    out[3] = 4.0 / (exp((-25.0 - V) / 5.0) + 1.0);
    /* alpha_n = 0.032 (-50 - V) / (exp((-50 - V)/5) - 1) */
    out[4] = 0.032 * 5.0 * xm1((-50.0 - V) / 5.0);
    /* beta_n  = 0.5 exp((-55 - V)/40) */
    out[5] = 0.5 * exp((-55.0 - V) / 40.0);
}

/* Ionic currents (pA) for conductances in nS and potentials in mV:
 * I_Na = gNa m^3 h (V - ENa), I_K = gK n^4 (V - EK), I_L = gL (V - EL). */
void oracle_hh_currents(const double p[7], double V, double m, double h, double n,
                        double out[3])
{
    /* p = {C, gNa, ENa, gK, EK, gL, EL} */
    out[0] = p[1] * m * m * m * h * (V - p[2]);
    out[1] = p[3] * n * n * n * n * (V - p[4]);
    out[2] = p[5] * (V - p[6]);
}

/* ------------------------------------------------------------------------ */
/* Network description, mirrored by the Python shim.                         */
/* ------------------------------------------------------------------------ */
enum { POP_HH = 0, POP_SOURCE = 1, POP_IZH = 2 };

typedef struct {
    int32_t kind;             /* POP_HH or POP_SOURCE */
    int32_t n;
    double C, gNa, ENa, gK, EK, gL, EL;     /* pF, nS, mV */
    double E_syn[2];          /* reversal potential of channel 0 / 1 (mV) */
    double tau_syn[2];        /* decay time constant of channel 0 / 1 (ms) */
    double v_thresh;          /* spike threshold (mV) */
    double src_rate_hz;       /* POP_SOURCE: Poisson rate */
    double drive_rate_hz;     /* POP_HH: rate of current-drive events (0 = none) */
    double drive_amp;         /* pA added per drive event */
    double drive_tau;         /* ms, decay of the drive current */
    const double* v0;         /* n initial potentials, or NULL for EL */
    /* POP_IZH (the cortical neuron model of ref. [9] of the paper, Sec. 5.1):
     * a = izh[0] + izh[1] r, b = izh[2] + izh[3] r, c = izh[4] + izh[5] r^2,
     * d = izh[6] + izh[7] r^2 with one uniform r per neuron; input current
     * bias + noise_sigma * z per step, z the Irwin-Hall normal of
     * oracle_izh_noise, plus the synaptic current g0 + g1 (current pulses). */
    double izh[8];
    double noise_sigma;
    double bias;
} oracle_pop;

typedef struct {
    int32_t pre, post;
    int32_t dense;            /* 0 = compressed rows, 1 = dense nPre x nPost */
    int32_t channel;          /* post conductance channel 0 / 1 */
    int64_t nnz;
    const int64_t* row_ptr;   /* nPre + 1 (rows) */
    const int32_t* col;       /* nnz (rows) */
    const double* w;          /* nnz (rows) or nPre*nPost row-major (dense) */
    double k1, k2, k3;        /* scaling law constants */
    double n_conn;            /* nConn fed to the law */
    double user_scale;        /* extra factor c */
} oracle_proj;

typedef struct {
    oracle_pop desc;
    uint32_t tag;             /* RNG tag: (instance << 8) | population */
    uint64_t thr_src, thr_drive;
    double dec[2], dec_drive;
    double *V, *m, *h, *n, *g[2], *iext, *isyn;
    int32_t* spk;             /* ascending spike list of the last step */
    int32_t nspk;
    int64_t spike_count;      /* spikes since creation */
    int64_t nan_count;        /* neuron-steps that ended with a NaN V */
} opop;

typedef struct {
    oracle_proj desc;
    int64_t* row_ptr;
    int32_t* col;
    double* w;
    double scale;             /* gScale * c */
} oproj;

typedef struct {
    int n_pops, n_projs, n_sub;
    double dt;
    uint64_t seed;
    uint32_t t;
    int64_t events;           /* synaptic events delivered (stored synapses of spiking rows) */
    opop* pops;
    oproj* projs;
} oracle_net;

void oracle_net_destroy(oracle_net* net);

static void* xcalloc(size_t n, size_t sz) { return calloc(n ? n : 1, sz); }

/* Gating steady state x_inf = alpha / (alpha + beta) at V. */
static void steady_gates(double V, double* m, double* h, double* n)
{
    double r[6];
    oracle_hh_rates(V, r);
    *m = r[0] / (r[0] + r[1]);
    *h = r[2] / (r[2] + r[3]);
    *n = r[4] / (r[4] + r[5]);
}

/* Creates a network.  Returns NULL on a bad description: projections out of
 * range, row starts not monotone, post indices out of range or not strictly
 * ascending in a row, or a scaling-law pole (nConn + k2 <= 0).  All arrays
 * are copied.  `instance` is folded into every RNG tag so that instance b of
 * a batch draws the same numbers as a stand-alone network created with b. */
oracle_net* oracle_net_create(const oracle_pop* pops, int n_pops, const oracle_proj* projs,
                              int n_projs, double dt, int n_sub, uint64_t seed, uint32_t instance)
{
    if (n_pops <= 0 || n_pops > 255 || n_projs < 0 || n_projs > 255 || !(dt > 0.0) || n_sub <= 0)
        return NULL;
    oracle_net* net = (oracle_net*)xcalloc(1, sizeof(oracle_net));
    net->n_pops = n_pops; net->n_projs = n_projs; net->n_sub = n_sub;
    net->dt = dt; net->seed = seed; net->t = 0;
    net->pops = (opop*)xcalloc((size_t)n_pops, sizeof(opop));
    net->projs = (oproj*)xcalloc((size_t)(n_projs ? n_projs : 1), sizeof(oproj));
    for (int p = 0; p < n_pops; ++p) {
        opop* P = &net->pops[p];
        P->desc = pops[p];
        P->desc.v0 = NULL;
        int n = pops[p].n;
        if (n < 0) { oracle_net_destroy(net); return NULL; }
        P->tag = (instance << 8) | (uint32_t)p;
        P->thr_src = oracle_bernoulli_threshold(pops[p].src_rate_hz * dt * 1e-3);
        P->thr_drive = oracle_bernoulli_threshold(pops[p].drive_rate_hz * dt * 1e-3);
        for (int c = 0; c < 2; ++c)
            P->dec[c] = pops[p].tau_syn[c] > 0.0 ? exp(-dt / pops[p].tau_syn[c]) : 0.0;
        P->dec_drive = pops[p].drive_tau > 0.0 ? exp(-dt / pops[p].drive_tau) : 0.0;
        P->V = (double*)xcalloc((size_t)n, sizeof(double));
        P->m = (double*)xcalloc((size_t)n, sizeof(double));
        P->h = (double*)xcalloc((size_t)n, sizeof(double));
        P->n = (double*)xcalloc((size_t)n, sizeof(double));
        P->g[0] = (double*)xcalloc((size_t)n, sizeof(double));
        P->g[1] = (double*)xcalloc((size_t)n, sizeof(double));
        P->iext = (double*)xcalloc((size_t)n, sizeof(double));
        P->isyn = (double*)xcalloc((size_t)n, sizeof(double));
        P->spk = (int32_t*)xcalloc((size_t)n, sizeof(int32_t));
        for (int i = 0; i < n; ++i) {
            double v = pops[p].v0 ? pops[p].v0[i] : pops[p].EL;
            P->V[i] = v;
            if (pops[p].kind == POP_HH) steady_gates(v, &P->m[i], &P->h[i], &P->n[i]);
            if (pops[p].kind == POP_IZH) {
                /* h holds the neuron's parameter draw r, m the recovery variable u = b v */
                double r = oracle_izh_r(seed, P->tag, (uint32_t)i);
                P->h[i] = r;
                P->m[i] = (pops[p].izh[2] + pops[p].izh[3] * r) * v;
            }
        }
    }
    for (int q = 0; q < n_projs; ++q) {
        oproj* Q = &net->projs[q];
        const oracle_proj* d = &projs[q];
        Q->desc = *d;
        if (d->pre < 0 || d->pre >= n_pops || d->post < 0 || d->post >= n_pops ||
            d->channel < 0 || d->channel > 1 || net->pops[d->post].desc.kind == POP_SOURCE) {
            oracle_net_destroy(net); return NULL;
        }
        double gs;
        if (oracle_gscale(d->k1, d->k2, d->k3, d->n_conn, &gs) != 0) {
            oracle_net_destroy(net); return NULL;
        }
        Q->scale = gs * d->user_scale;
        int64_t n_pre = pops[d->pre].n, n_post = pops[d->post].n;
        if (d->dense) {
            Q->w = (double*)xcalloc((size_t)(n_pre * n_post), sizeof(double));
            memcpy(Q->w, d->w, (size_t)(n_pre * n_post) * sizeof(double));
        } else {
            if (d->row_ptr[0] != 0 || d->row_ptr[n_pre] != d->nnz) { oracle_net_destroy(net); return NULL; }
            for (int64_t i = 0; i < n_pre; ++i) {
                if (d->row_ptr[i + 1] < d->row_ptr[i]) { oracle_net_destroy(net); return NULL; }
                for (int64_t k = d->row_ptr[i]; k < d->row_ptr[i + 1]; ++k) {
                    if (d->col[k] < 0 || d->col[k] >= n_post) { oracle_net_destroy(net); return NULL; }
                    if (k > d->row_ptr[i] && d->col[k] <= d->col[k - 1]) { oracle_net_destroy(net); return NULL; }
                }
            }
            Q->row_ptr = (int64_t*)xcalloc((size_t)(n_pre + 1), sizeof(int64_t));
            Q->col = (int32_t*)xcalloc((size_t)d->nnz, sizeof(int32_t));
            Q->w = (double*)xcalloc((size_t)d->nnz, sizeof(double));
            memcpy(Q->row_ptr, d->row_ptr, (size_t)(n_pre + 1) * sizeof(int64_t));
            memcpy(Q->col, d->col, (size_t)d->nnz * sizeof(int32_t));
            memcpy(Q->w, d->w, (size_t)d->nnz * sizeof(double));
        }
        Q->desc.row_ptr = NULL; Q->desc.col = NULL; Q->desc.w = NULL;
    }
    return net;
}

void oracle_net_destroy(oracle_net* net)
{
    if (!net) return;
    for (int p = 0; p < net->n_pops; ++p) {
        opop* P = &net->pops[p];
        free(P->V); free(P->m); free(P->h); free(P->n); free(P->g[0]); free(P->g[1]);
        free(P->iext); free(P->isyn); free(P->spk);
    }
    for (int q = 0; q < net->n_projs; ++q) {
        free(net->projs[q].row_ptr); free(net->projs[q].col); free(net->projs[q].w);
    }
    free(net->pops); free(net->projs); free(net);
}

double oracle_net_scale(const oracle_net* net, int proj) { return net->projs[proj].scale; }
uint32_t oracle_net_time(const oracle_net* net) { return net->t; }
int64_t oracle_net_events(const oracle_net* net) { return net->events; }

/* One Euler substep of the HH equations for a single neuron. */
static void hh_substep(const oracle_pop* d, double hs, double I_in,
                       double* V, double* m, double* h, double* n)
{
    double r[6], I[3];
    const double p[7] = {d->C, d->gNa, d->ENa, d->gK, d->EK, d->gL, d->EL};
    oracle_hh_rates(*V, r);
    oracle_hh_currents(p, *V, *m, *h, *n, I);
    double dV = (I_in - I[0] - I[1] - I[2]) / d->C;
    double dm = r[0] * (1.0 - *m) - r[1] * *m;
    double dh = r[2] * (1.0 - *h) - r[3] * *h;
    double dn = r[4] * (1.0 - *n) - r[5] * *n;
    *V += hs * dV; *m += hs * dm; *h += hs * dh; *n += hs * dn;
}

/* Threads of oracle_net_step (timing only; default 1).  With one thread the
 * step is the plain sequential loop.  With more, neurons are updated in a
 * parallel loop (each neuron's arithmetic unchanged, spike lists compacted
 * in index order afterwards), dense rows are delivered by post ranges (the
 * per-post summation order unchanged) and compressed rows by spike ranges
 * into per-thread accumulators added in thread order, which changes the
 * order of the floating-point sums of compressed-row events. */
static int g_threads = 1;
void oracle_set_threads(int n) { g_threads = n < 1 ? 1 : n; }
int oracle_get_threads(void) { return g_threads; }

/* The per-neuron update of population P at step t; returns 1 on a spike
 * and sets *nan when V ends as NaN. */
static int neuron_update(const oracle_net* net, opop* P, int i, uint32_t t, double hs, int* nan)
{
    const oracle_pop* d = &P->desc;
    *nan = 0;
    if (d->kind == POP_SOURCE) {
        uint32_t u = draw_u32(net->seed, (uint32_t)i, t, P->tag, STREAM_SOURCE, 0);
        return (uint64_t)u < P->thr_src;
    }
    if (d->kind == POP_IZH) {
        /* Ref. [9]: v' = 0.04 v^2 + 5 v + 140 - u + I, u' = a (b v - u);
         * v >= v_thresh (30 mV) fires and resets v <- c, u <- u + d.
         * v takes n_sub Euler substeps of dt / n_sub, then u one step of dt
         * with the new v, as in the model's published scheme. */
        const double r = P->h[i];
        const double a = d->izh[0] + d->izh[1] * r, b = d->izh[2] + d->izh[3] * r;
        const double c = d->izh[4] + d->izh[5] * r * r, dd = d->izh[6] + d->izh[7] * r * r;
        const double isyn = P->g[0][i] + P->g[1][i];
        const double I = d->bias + d->noise_sigma * oracle_izh_noise(net->seed, P->tag, t, (uint32_t)i) + isyn;
        P->isyn[i] = isyn;
        double v = P->V[i], u = P->m[i];
        for (int s = 0; s < net->n_sub; ++s) v += hs * (0.04 * v * v + 5.0 * v + 140.0 - u + I);
        u += net->dt * a * (b * v - u);
        int spike = 0;
        if (v >= d->v_thresh) {
            spike = 1;
            v = c;
            u += dd;
        }
        *nan = isnan(v) ? 1 : 0;
        P->V[i] = v;
        P->m[i] = u;
        P->g[0][i] *= P->dec[0];
        P->g[1][i] *= P->dec[1];
        return spike;
    }
    if (P->thr_drive) {
        uint32_t u = draw_u32(net->seed, (uint32_t)i, t, P->tag, STREAM_DRIVE, 0);
        if ((uint64_t)u < P->thr_drive) P->iext[i] += d->drive_amp;
    }
    double V0 = P->V[i];
    double isyn = P->g[0][i] * (d->E_syn[0] - V0) + P->g[1][i] * (d->E_syn[1] - V0);
    P->isyn[i] = isyn;
    double V = V0, m = P->m[i], h = P->h[i], n = P->n[i];
    for (int s = 0; s < net->n_sub; ++s) hh_substep(d, hs, isyn + P->iext[i], &V, &m, &h, &n);
    P->V[i] = V; P->m[i] = m; P->h[i] = h; P->n[i] = n;
    *nan = isnan(V) ? 1 : 0;
    P->g[0][i] *= P->dec[0];
    P->g[1][i] *= P->dec[1];
    P->iext[i] *= P->dec_drive;
    return V0 < d->v_thresh && V >= d->v_thresh;
}

/* One time step of dt, in this order (Izhikevich populations: see
 * neuron_update; their synaptic input is the current g0 + g1):
 *   1. Poisson sources draw their spikes;
 *   2. driven HH neurons draw a drive event and add drive_amp to I_ext;
 *   3. I_syn = sum_c g_c (E_c - V) from step-start state;
 *   4. n_sub Euler substeps of V, m, h, n with I_syn + I_ext held;
 *   5. spike where V crossed v_thresh upward, listed in ascending index;
 *   6. conductances and drive current decay by exp(-dt / tau);
 *   7. every spike of this step adds scale * w to the post conductances. */
void oracle_net_step(oracle_net* net)
{
    const uint32_t t = net->t;
    const double hs = net->dt / net->n_sub;
    const int nt = g_threads;
    for (int p = 0; p < net->n_pops; ++p) {
        opop* P = &net->pops[p];
        const int n = P->desc.n;
        P->nspk = 0;
        if (nt == 1) {
            for (int i = 0; i < n; ++i) {
                int nan;
                if (neuron_update(net, P, i, t, hs, &nan)) P->spk[P->nspk++] = i;
                P->nan_count += nan;
            }
        } else {
            /* flags in the spike-list buffer (1 spike, 2 NaN), compacted after */
            int64_t nans = 0;
            #pragma omp parallel for num_threads(nt) schedule(static) reduction(+:nans)
            for (int i = 0; i < n; ++i) {
                int nan;
                const int s = neuron_update(net, P, i, t, hs, &nan);
                P->spk[i] = s;
                nans += nan;
            }
            for (int i = 0; i < n; ++i)
                if (P->spk[i]) P->spk[P->nspk++] = i;
            P->nan_count += nans;
        }
        P->spike_count += P->nspk;
    }
    for (int q = 0; q < net->n_projs; ++q) {
        const oproj* Q = &net->projs[q];
        const opop* pre = &net->pops[Q->desc.pre];
        double* g = net->pops[Q->desc.post].g[Q->desc.channel];
        int64_t n_post = net->pops[Q->desc.post].desc.n;
        if (Q->desc.dense) {
            if (nt == 1) {
                for (int s = 0; s < pre->nspk; ++s) {
                    const int64_t i = pre->spk[s];
                    for (int64_t j = 0; j < n_post; ++j) g[j] += Q->scale * Q->w[i * n_post + j];
                }
            } else {
                #pragma omp parallel for num_threads(nt) schedule(static)
                for (int64_t j = 0; j < n_post; ++j)
                    for (int s = 0; s < pre->nspk; ++s)
                        g[j] += Q->scale * Q->w[(int64_t)pre->spk[s] * n_post + j];
            }
            net->events += (int64_t)pre->nspk * n_post;
        } else {
            int64_t ev = 0;
            for (int s = 0; s < pre->nspk; ++s) ev += Q->row_ptr[pre->spk[s] + 1] - Q->row_ptr[pre->spk[s]];
            if (nt == 1 || ev < 4096) {
                for (int s = 0; s < pre->nspk; ++s) {
                    const int64_t i = pre->spk[s];
                    for (int64_t k = Q->row_ptr[i]; k < Q->row_ptr[i + 1]; ++k) g[Q->col[k]] += Q->scale * Q->w[k];
                }
            } else {
                double* buf = (double*)xcalloc((size_t)(nt * n_post), sizeof(double));
                #pragma omp parallel num_threads(nt)
                {
                    int th = 0;
#ifdef _OPENMP
                    th = omp_get_thread_num();
#endif
                    double* mine = buf + (size_t)th * n_post;
                    #pragma omp for schedule(static)
                    for (int s = 0; s < pre->nspk; ++s) {
                        const int64_t i = pre->spk[s];
                        for (int64_t k = Q->row_ptr[i]; k < Q->row_ptr[i + 1]; ++k)
                            mine[Q->col[k]] += Q->scale * Q->w[k];
                    }
                    #pragma omp for schedule(static)
                    for (int64_t j = 0; j < n_post; ++j)
                        for (int u = 0; u < nt; ++u) g[j] += buf[(size_t)u * n_post + j];
                }
                free(buf);
            }
            net->events += ev;
        }
    }
    net->t = t + 1;
}

void oracle_net_run(oracle_net* net, int64_t n_steps)
{
    for (int64_t s = 0; s < n_steps; ++s) oracle_net_step(net);
}

/* Field access.  field: 0 V, 1 m, 2 h, 3 n, 4 g0, 5 g1, 6 I_ext, 7 I_syn of
 * the last step. */
static double* field_ptr(opop* P, int field)
{
    switch (field) {
    case 0: return P->V; case 1: return P->m; case 2: return P->h; case 3: return P->n;
    case 4: return P->g[0]; case 5: return P->g[1]; case 6: return P->iext; case 7: return P->isyn;
    default: return NULL;
    }
}

int oracle_net_get(oracle_net* net, int pop, int field, double* out)
{
    if (pop < 0 || pop >= net->n_pops) return -1;
    double* f = field_ptr(&net->pops[pop], field);
    if (!f) return -1;
    memcpy(out, f, (size_t)net->pops[pop].desc.n * sizeof(double));
    return 0;
}

int oracle_net_set(oracle_net* net, int pop, int field, const double* in)
{
    if (pop < 0 || pop >= net->n_pops) return -1;
    double* f = field_ptr(&net->pops[pop], field);
    if (!f || field == 7) return -1;
    memcpy(f, in, (size_t)net->pops[pop].desc.n * sizeof(double));
    return 0;
}

/* Ascending spike list of the last step; returns its length. */
int32_t oracle_net_spikes(const oracle_net* net, int pop, int32_t* out)
{
    const opop* P = &net->pops[pop];
    if (out) memcpy(out, P->spk, (size_t)P->nspk * sizeof(int32_t));
    return P->nspk;
}

void oracle_net_counters(const oracle_net* net, int pop, int64_t* spike_count, int64_t* nan_count)
{
    *spike_count = net->pops[pop].spike_count;
    *nan_count = net->pops[pop].nan_count;
}

/* Adds the events of the given spike list of projection q's pre population
 * to its post conductances, exactly as step 7 does. */
void oracle_net_deliver(oracle_net* net, int q, const int32_t* spk, int32_t nspk)
{
    const oproj* Q = &net->projs[q];
    double* g = net->pops[Q->desc.post].g[Q->desc.channel];
    int64_t n_post = net->pops[Q->desc.post].desc.n;
    for (int s = 0; s < nspk; ++s) {
        int64_t i = spk[s];
        if (Q->desc.dense) {
            for (int64_t j = 0; j < n_post; ++j) g[j] += Q->scale * Q->w[i * n_post + j];
        } else {
            for (int64_t k = Q->row_ptr[i]; k < Q->row_ptr[i + 1]; ++k) g[Q->col[k]] += Q->scale * Q->w[k];
        }
    }
}

/* Event list of a spike list over compressed rows: for each spike in list
 * order, the (post index, weight) pairs of its row in storage order.
 * Returns the number of events; out arrays may be NULL to only count. */
int64_t oracle_event_list(const int64_t* row_ptr, const int32_t* col, const double* w,
                          const int32_t* spk, int32_t nspk, int32_t* post_out, double* w_out)
{
    int64_t e = 0;
    for (int s = 0; s < nspk; ++s) {
        int64_t i = spk[s];
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k, ++e) {
            if (post_out) post_out[e] = col[k];
            if (w_out) w_out[e] = w[k];
        }
    }
    return e;
}

/* ------------------------------------------------------------------------ */
/* Compressed-row connectivity drawn from the seed: one Bernoulli(p) draw   */
/* per (pre i, post j) pair, Philox counter (j / 4, i, tag, STREAM_CSR) and */
/* output word j % 4; post indices ascend within a row (Sec. 3 layout).     */
/* ------------------------------------------------------------------------ */
static int csr_edge(uint64_t seed, uint32_t tag, uint64_t thr, int64_t i, int64_t j)
{
    uint32_t u = draw_u32(seed, (uint32_t)(j >> 2), (uint32_t)i, tag, STREAM_CSR, (int)(j & 3));
    return (uint64_t)u < thr;
}

/* Fills row_ptr[n_pre + 1] and returns nnz. */
int64_t oracle_csr_rows(uint64_t seed, uint32_t tag, int64_t n_pre, int64_t n_post, double p,
                        int64_t* row_ptr)
{
    uint64_t thr = oracle_bernoulli_threshold(p);
    row_ptr[0] = 0;
    for (int64_t i = 0; i < n_pre; ++i) {
        int64_t c = 0;
        for (int64_t j = 0; j < n_post; ++j) c += csr_edge(seed, tag, thr, i, j);
        row_ptr[i + 1] = row_ptr[i] + c;
    }
    return row_ptr[n_pre];
}

void oracle_csr_fill(uint64_t seed, uint32_t tag, int64_t n_pre, int64_t n_post, double p,
                     const int64_t* row_ptr, int32_t* col)
{
    uint64_t thr = oracle_bernoulli_threshold(p);
    for (int64_t i = 0; i < n_pre; ++i) {
        int64_t k = row_ptr[i];
        for (int64_t j = 0; j < n_post; ++j)
            if (csr_edge(seed, tag, thr, i, j)) col[k++] = (int32_t)j;
    }
}

/* Poisson source draw for neuron i of a population with RNG tag `tag` at
 * step t: 1 when the 32-bit draw is below round(rate * dt * 2^32). */
int oracle_source_spike(uint64_t seed, uint32_t tag, uint32_t t, uint32_t i, double rate_hz, double dt)
{
    uint32_t u = draw_u32(seed, i, t, tag, STREAM_SOURCE, 0);
    return (uint64_t)u < oracle_bernoulli_threshold(rate_hz * dt * 1e-3);
}
