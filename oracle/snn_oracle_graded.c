/*
 * FP64 oracle of the differentiable (graded-synapse) form and its gradient.
 *
 * TEST INFRASTRUCTURE ONLY (see snn_oracle.c).  Shares no source with the
 * CUDA library.
 *
 * The network is the HH network of Sec. 2 with graded instead of spiking
 * synapses (a reading: the paper does not fix the synapse model).  Each step:
 *   1. drive events of driven populations (I_ext += A, Philox draw < round(p 2^32));
 *   2. release r_i = 1 / (1 + exp((v_thr - V_i) / slope)) of every pre neuron;
 *   3. G_q[k] = sum_i w_ik r_i for every projection q (compressed rows, Sec. 3);
 *   4. I_syn_k = sum_q s_q (E_{post, channel q} - V_k) G_q[k], s_q = gScale * c (Sec. 5.1);
 *   5. n_sub forward-Euler substeps of V, m, h, n with I_syn + I_ext held;
 *   6. I_ext decays; the output population's filter y += (dt / tau_f)(V - y);
 *   7. loss += sum over outputs of (y - target_t)^2; L = loss / (T * N_out).
 * The gradient of L with respect to every s_q and w_ik is the discrete adjoint
 * of exactly these operations (reverse sweep over stored step states, with
 * the substeps recomputed), written from the chain rule.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "oracle_internal.h"

typedef struct {
    int32_t n;
    double C, gNa, ENa, gK, EK, gL, EL;
    double E_syn[2];
    double drive_rate_hz, drive_amp, drive_tau;
    const double* v0;
} oracle_gpop;

typedef struct {
    int32_t pre, post, channel;
    int64_t nnz;
    const int64_t* row_ptr;
    const int32_t* col;
    const double* w;
    double k1, k2, k3, n_conn, user_scale;
    double v_thr, v_slope;
} oracle_gproj;

typedef struct {
    oracle_gpop d;
    double* v0;                 /* owned copy of the initial potentials */
    uint32_t tag;
    uint64_t thr_drive;
    double dec_drive;
    int off;                    /* offset in the concatenated neuron arrays */
} gpop;

typedef struct {
    oracle_gproj d;
    int64_t* row_ptr;
    int32_t* col;
    double* w;
    double scale;
} gproj;

typedef struct {
    int n_pops, n_projs, n_sub, out_pop, N;
    double dt, tau_f;
    uint64_t seed;
    gpop* pops;
    gproj* projs;
    int* pop_of;                /* neuron -> population */
    /* recorded forward: T + 1 step-start states and T steps of G and releases */
    int T;
    double *V, *m, *h, *n, *ie, *y;   /* [(T + 1) * N] (y only meaningful for outputs) */
    double* G;                  /* [T * sum over projections of n_post] */
    int64_t* g_off;             /* per projection offset of its G block within one step */
    int64_t g_step;             /* floats of G per step */
    double* target;             /* [T * N_out] */
    double loss;
} graded_net;

static void* xc(size_t n, size_t s) { return calloc(n ? n : 1, s); }

void oracle_graded_destroy(graded_net* g)
{
    if (!g) return;
    for (int q = 0; q < g->n_projs; ++q) { free(g->projs[q].row_ptr); free(g->projs[q].col); free(g->projs[q].w); }
    for (int p = 0; p < g->n_pops; ++p) free(g->pops[p].v0);
    free(g->pops); free(g->projs); free(g->pop_of);
    free(g->V); free(g->m); free(g->h); free(g->n); free(g->ie); free(g->y);
    free(g->G); free(g->g_off); free(g->target);
    free(g);
}

graded_net* oracle_graded_create(const oracle_gpop* pops, int n_pops, const oracle_gproj* projs, int n_projs,
                                 double dt, int n_sub, uint64_t seed, uint32_t instance, int out_pop,
                                 double tau_f)
{
    if (n_pops <= 0 || n_pops > 255 || n_projs < 0 || !(dt > 0) || n_sub <= 0 || out_pop < 0 ||
        out_pop >= n_pops || !(tau_f > 0))
        return NULL;
    graded_net* g = (graded_net*)xc(1, sizeof(graded_net));
    g->n_pops = n_pops; g->n_projs = n_projs; g->n_sub = n_sub; g->out_pop = out_pop;
    g->dt = dt; g->tau_f = tau_f; g->seed = seed;
    g->pops = (gpop*)xc((size_t)n_pops, sizeof(gpop));
    g->projs = (gproj*)xc((size_t)n_projs, sizeof(gproj));
    int off = 0;
    for (int p = 0; p < n_pops; ++p) {
        g->pops[p].d = pops[p];
        g->pops[p].d.v0 = NULL;
        g->pops[p].v0 = (double*)xc((size_t)(pops[p].n > 0 ? pops[p].n : 1), sizeof(double));
        for (int i = 0; i < pops[p].n; ++i) g->pops[p].v0[i] = pops[p].v0 ? pops[p].v0[i] : pops[p].EL;
        g->pops[p].tag = (instance << 8) | (uint32_t)p;
        g->pops[p].thr_drive = oracle_bernoulli_threshold(pops[p].drive_rate_hz * dt * 1e-3);
        g->pops[p].dec_drive = pops[p].drive_tau > 0 ? exp(-dt / pops[p].drive_tau) : 0.0;
        g->pops[p].off = off;
        off += pops[p].n;
    }
    g->N = off;
    g->pop_of = (int*)xc((size_t)off, sizeof(int));
    for (int p = 0; p < n_pops; ++p)
        for (int i = 0; i < pops[p].n; ++i) g->pop_of[g->pops[p].off + i] = p;
    g->g_off = (int64_t*)xc((size_t)n_projs, sizeof(int64_t));
    g->g_step = 0;
    for (int q = 0; q < n_projs; ++q) {
        const oracle_gproj* d = &projs[q];
        gproj* Q = &g->projs[q];
        if (d->pre < 0 || d->pre >= n_pops || d->post < 0 || d->post >= n_pops || d->channel < 0 ||
            d->channel > 1 || !(d->v_slope > 0)) { oracle_graded_destroy(g); return NULL; }
        double gs;
        if (oracle_gscale(d->k1, d->k2, d->k3, d->n_conn, &gs) != 0) { oracle_graded_destroy(g); return NULL; }
        Q->d = *d;
        Q->scale = gs * d->user_scale;
        int64_t n_pre = pops[d->pre].n;
        Q->row_ptr = (int64_t*)xc((size_t)(n_pre + 1), sizeof(int64_t));
        Q->col = (int32_t*)xc((size_t)d->nnz, sizeof(int32_t));
        Q->w = (double*)xc((size_t)d->nnz, sizeof(double));
        memcpy(Q->row_ptr, d->row_ptr, (size_t)(n_pre + 1) * sizeof(int64_t));
        memcpy(Q->col, d->col, (size_t)d->nnz * sizeof(int32_t));
        memcpy(Q->w, d->w, (size_t)d->nnz * sizeof(double));
        Q->d.row_ptr = NULL; Q->d.col = NULL; Q->d.w = NULL;
        g->g_off[q] = g->g_step;
        g->g_step += pops[d->post].n;
    }
    return g;
}

double oracle_graded_get_scale(graded_net* g, int q) { return g->projs[q].scale; }
void oracle_graded_set_scale(graded_net* g, int q, double s) { g->projs[q].scale = s; }
void oracle_graded_set_weight(graded_net* g, int q, int64_t k, double w) { g->projs[q].w[k] = w; }
double oracle_graded_get_weight(graded_net* g, int q, int64_t k) { return g->projs[q].w[k]; }

static double release(double V, double v_thr, double slope) { return 1.0 / (1.0 + exp((v_thr - V) / slope)); }

/* x / (exp(x) - 1) and its derivative in x. */
static double lin(double x)
{
    if (fabs(x) < 1e-6) return 1.0 - 0.5 * x + x * x / 12.0;
    return x / expm1(x);
}
static double dlin(double x)
{
    if (fabs(x) < 1e-4) return -0.5 + x / 6.0 - x * x * x / 180.0;
    double em = expm1(x);
    return (em - x * (em + 1.0)) / (em * em);
}

/* Derivatives in V of the six Traub-Miles rates (same order as oracle_hh_rates). */
void oracle_hh_rate_derivs(double V, double out[6])
{
    out[0] = 0.32 * 4.0 * dlin((-52.0 - V) / 4.0) * (-0.25);
    out[1] = 0.28 * 5.0 * dlin((V + 25.0) / 5.0) * 0.2;
    out[2] = -0.128 * exp((-48.0 - V) / 18.0) / 18.0;
    double u = exp((-25.0 - V) / 5.0);
    out[3] = 4.0 * u / ((u + 1.0) * (u + 1.0)) / 5.0;
    out[4] = 0.032 * 5.0 * dlin((-50.0 - V) / 5.0) * (-0.2);
    out[5] = -0.5 * exp((-55.0 - V) / 40.0) / 40.0;
    (void)lin;
}

/* Runs T steps from the initial state, recording every step-start state and
 * every G, and returns L.  target: T * N_out values (mV); y_out may be NULL. */
double oracle_graded_forward(graded_net* g, int T, const double* target, double* y_out)
{
    const int N = g->N;
    const gpop* OP = &g->pops[g->out_pop];
    const int n_out = OP->d.n;
    free(g->V); free(g->m); free(g->h); free(g->n); free(g->ie); free(g->y); free(g->G); free(g->target);
    g->T = T;
    size_t S = (size_t)(T + 1) * N;
    g->V = (double*)xc(S, sizeof(double)); g->m = (double*)xc(S, sizeof(double));
    g->h = (double*)xc(S, sizeof(double)); g->n = (double*)xc(S, sizeof(double));
    g->ie = (double*)xc(S, sizeof(double)); g->y = (double*)xc(S, sizeof(double));
    g->G = (double*)xc((size_t)T * (size_t)g->g_step, sizeof(double));
    g->target = (double*)xc((size_t)T * n_out, sizeof(double));
    memcpy(g->target, target, (size_t)T * n_out * sizeof(double));
    for (int p = 0; p < g->n_pops; ++p) {
        const gpop* P = &g->pops[p];
        for (int i = 0; i < P->d.n; ++i) {
            double v = P->v0[i], r[6];
            oracle_hh_rates(v, r);
            int k = P->off + i;
            g->V[k] = v;
            g->m[k] = r[0] / (r[0] + r[1]); g->h[k] = r[2] / (r[2] + r[3]); g->n[k] = r[4] / (r[4] + r[5]);
            g->ie[k] = 0.0;
            g->y[k] = v;
        }
    }
    const uint32_t key[2] = {(uint32_t)(g->seed & 0xffffffffu), (uint32_t)(g->seed >> 32)};
    const double hs = g->dt / g->n_sub, a = g->dt / g->tau_f;
    double loss = 0.0;
    double* ie_now = (double*)xc((size_t)N, sizeof(double));
    double* rel = (double*)xc((size_t)N, sizeof(double));
    for (int t = 0; t < T; ++t) {
        const double* V0 = g->V + (size_t)t * N;
        double* G = g->G + (size_t)t * g->g_step;
        /* 1. drive events */
        for (int p = 0; p < g->n_pops; ++p) {
            const gpop* P = &g->pops[p];
            for (int i = 0; i < P->d.n; ++i) {
                int k = P->off + i;
                double ie = g->ie[(size_t)t * N + k];
                if (P->thr_drive) {
                    uint32_t ctr[4] = {(uint32_t)i, (uint32_t)t, P->tag, 2u}, out[4];
                    oracle_philox4x32_10(ctr, key, out);
                    if ((uint64_t)out[0] < P->thr_drive) ie += P->d.drive_amp;
                }
                ie_now[k] = ie;
            }
        }
        /* 2-3. releases and graded conductances, per projection */
        for (int q = 0; q < g->n_projs; ++q) {
            const gproj* Q = &g->projs[q];
            const gpop* pre = &g->pops[Q->d.pre];
            double* Gq = G + g->g_off[q];
            for (int i = 0; i < pre->d.n; ++i) rel[i] = release(V0[pre->off + i], Q->d.v_thr, Q->d.v_slope);
            for (int i = 0; i < pre->d.n; ++i)
                for (int64_t e = Q->row_ptr[i]; e < Q->row_ptr[i + 1]; ++e) Gq[Q->col[e]] += Q->w[e] * rel[i];
        }
        /* 4-6. neuron update */
        for (int p = 0; p < g->n_pops; ++p) {
            const gpop* P = &g->pops[p];
            const double prm[7] = {P->d.C, P->d.gNa, P->d.ENa, P->d.gK, P->d.EK, P->d.gL, P->d.EL};
            for (int i = 0; i < P->d.n; ++i) {
                int k = P->off + i;
                size_t s0 = (size_t)t * N + k, s1 = (size_t)(t + 1) * N + k;
                double V = V0[k], m = g->m[s0], h = g->h[s0], n = g->n[s0];
                double isyn = 0.0;
                for (int q = 0; q < g->n_projs; ++q) {
                    const gproj* Q = &g->projs[q];
                    if (Q->d.post != p) continue;
                    isyn += Q->scale * (P->d.E_syn[Q->d.channel] - V) * G[g->g_off[q] + i];
                }
                double I_in = isyn + ie_now[k];
                for (int sub = 0; sub < g->n_sub; ++sub) {
                    double r[6], I[3];
                    oracle_hh_rates(V, r);
                    oracle_hh_currents(prm, V, m, h, n, I);
                    double dV = (I_in - I[0] - I[1] - I[2]) / P->d.C;
                    double dm = r[0] * (1 - m) - r[1] * m, dh = r[2] * (1 - h) - r[3] * h, dn = r[4] * (1 - n) - r[5] * n;
                    V += hs * dV; m += hs * dm; h += hs * dh; n += hs * dn;
                }
                g->V[s1] = V; g->m[s1] = m; g->h[s1] = h; g->n[s1] = n;
                g->ie[s1] = ie_now[k] * P->dec_drive;
                g->y[s1] = g->y[s0] + a * (V - g->y[s0]);
            }
        }
        /* 7. loss on the output filter */
        for (int i = 0; i < n_out; ++i) {
            double y = g->y[(size_t)(t + 1) * N + OP->off + i];
            double d = y - target[(size_t)t * n_out + i];
            loss += d * d;
            if (y_out) y_out[(size_t)t * n_out + i] = y;
        }
    }
    free(ie_now); free(rel);
    g->loss = loss / ((double)T * n_out);
    return g->loss;
}

/* Reverse sweep: grad_scale[q] and grad_w[q][e] (compressed-row order) of a
 * loss whose gradient with respect to the output filter is dL_dy[t][i] =
 * dL / dy_i(t + 1) (T * N_out values); NULL takes the squared-error loss L of
 * the forward pass, dL_dy = 2 (y - target) / (T * N_out). */
static int graded_backward(graded_net* g, const double* dL_dy, double* grad_scale, double** grad_w)
{
    if (!g->V || g->T <= 0) return -1;
    const int N = g->N, T = g->T;
    const gpop* OP = &g->pops[g->out_pop];
    const int n_out = OP->d.n;
    const double hs = g->dt / g->n_sub, a = g->dt / g->tau_f;
    const double nrm = 2.0 / ((double)T * n_out);
    for (int q = 0; q < g->n_projs; ++q) {
        grad_scale[q] = 0.0;
        memset(grad_w[q], 0, (size_t)g->projs[q].d.nnz * sizeof(double));
    }
    /* adjoints of the state at the end of the current step */
    double *lV = (double*)xc((size_t)N, sizeof(double)), *lm = (double*)xc((size_t)N, sizeof(double));
    double *lh = (double*)xc((size_t)N, sizeof(double)), *ln = (double*)xc((size_t)N, sizeof(double));
    double *ly = (double*)xc((size_t)N, sizeof(double));
    double *nV = (double*)xc((size_t)N, sizeof(double)), *mu = (double*)xc((size_t)N, sizeof(double));
    double* nu = (double*)xc((size_t)g->g_step, sizeof(double));
    double* ie_now = (double*)xc((size_t)N, sizeof(double));
    const uint32_t key[2] = {(uint32_t)(g->seed & 0xffffffffu), (uint32_t)(g->seed >> 32)};
    for (int t = T - 1; t >= 0; --t) {
        const double* V0 = g->V + (size_t)t * N;
        const double* G = g->G + (size_t)t * g->g_step;
        /* loss term of step t on y(t + 1) */
        for (int i = 0; i < n_out; ++i) {
            int k = OP->off + i;
            if (dL_dy)
                ly[k] += dL_dy[(size_t)t * n_out + i];
            else
                ly[k] += nrm * (g->y[(size_t)(t + 1) * N + k] - g->target[(size_t)t * n_out + i]);
        }
        /* drive current of this step (recomputed, it holds no parameter) */
        for (int p = 0; p < g->n_pops; ++p) {
            const gpop* P = &g->pops[p];
            for (int i = 0; i < P->d.n; ++i) {
                int k = P->off + i;
                double ie = g->ie[(size_t)t * N + k];
                if (P->thr_drive) {
                    uint32_t ctr[4] = {(uint32_t)i, (uint32_t)t, P->tag, 2u}, out[4];
                    oracle_philox4x32_10(ctr, key, out);
                    if ((uint64_t)out[0] < P->thr_drive) ie += P->d.drive_amp;
                }
                ie_now[k] = ie;
            }
        }
        /* neuron part: back through the filter and the substeps */
        for (int p = 0; p < g->n_pops; ++p) {
            const gpop* P = &g->pops[p];
            const double prm[7] = {P->d.C, P->d.gNa, P->d.ENa, P->d.gK, P->d.EK, P->d.gL, P->d.EL};
            for (int i = 0; i < P->d.n; ++i) {
                int k = P->off + i;
                size_t s0 = (size_t)t * N + k;
                /* y(t+1) = y(t) + a (V(t+1) - y(t)) */
                double lVend = lV[k] + (p == g->out_pop ? a * ly[k] : 0.0);
                double ly_prev = (p == g->out_pop) ? (1.0 - a) * ly[k] : 0.0;
                double isyn = 0.0, dIsyn_dV = 0.0;
                for (int q = 0; q < g->n_projs; ++q) {
                    const gproj* Q = &g->projs[q];
                    if (Q->d.post != p) continue;
                    double Gq = G[g->g_off[q] + i];
                    isyn += Q->scale * (P->d.E_syn[Q->d.channel] - V0[k]) * Gq;
                    dIsyn_dV -= Q->scale * Gq;
                }
                double I_in = isyn + ie_now[k];
                /* recompute the substep states */
                double Vs[65], ms[65], hsv[65], ns[65];
                int S = g->n_sub;
                Vs[0] = V0[k]; ms[0] = g->m[s0]; hsv[0] = g->h[s0]; ns[0] = g->n[s0];
                for (int s = 0; s < S; ++s) {
                    double r[6], I[3];
                    oracle_hh_rates(Vs[s], r);
                    oracle_hh_currents(prm, Vs[s], ms[s], hsv[s], ns[s], I);
                    Vs[s + 1] = Vs[s] + hs * (I_in - I[0] - I[1] - I[2]) / P->d.C;
                    ms[s + 1] = ms[s] + hs * (r[0] * (1 - ms[s]) - r[1] * ms[s]);
                    hsv[s + 1] = hsv[s] + hs * (r[2] * (1 - hsv[s]) - r[3] * hsv[s]);
                    ns[s + 1] = ns[s] + hs * (r[4] * (1 - ns[s]) - r[5] * ns[s]);
                }
                double aV = lVend, am = lm[k], ah = lh[k], an = ln[k], aI = 0.0;
                for (int s = S - 1; s >= 0; --s) {
                    double V = Vs[s], m = ms[s], h = hsv[s], n = ns[s], r[6], dr[6];
                    oracle_hh_rates(V, r);
                    oracle_hh_rate_derivs(V, dr);
                    double m3 = m * m * m, n3 = n * n * n;
                    double dI_dV = P->d.gNa * m3 * h + P->d.gK * n3 * n + P->d.gL;
                    double dI_dm = 3.0 * P->d.gNa * m * m * h * (V - P->d.ENa);
                    double dI_dh = P->d.gNa * m3 * (V - P->d.ENa);
                    double dI_dn = 4.0 * P->d.gK * n3 * (V - P->d.EK);
                    double c = hs / P->d.C;
                    double nV_ = aV * (1.0 - c * dI_dV) + am * hs * (dr[0] * (1 - m) - dr[1] * m) +
                                 ah * hs * (dr[2] * (1 - h) - dr[3] * h) + an * hs * (dr[4] * (1 - n) - dr[5] * n);
                    double nm_ = aV * (-c * dI_dm) + am * (1.0 - hs * (r[0] + r[1]));
                    double nh_ = aV * (-c * dI_dh) + ah * (1.0 - hs * (r[2] + r[3]));
                    double nn_ = aV * (-c * dI_dn) + an * (1.0 - hs * (r[4] + r[5]));
                    aI += aV * c;
                    aV = nV_; am = nm_; ah = nh_; an = nn_;
                }
                mu[k] = aI;                       /* dL / dI_syn of this step */
                nV[k] = aV + aI * dIsyn_dV;       /* pre-synaptic gather added below */
                lm[k] = am; lh[k] = ah; ln[k] = an;
                ly[k] = ly_prev;
                for (int q = 0; q < g->n_projs; ++q) {
                    const gproj* Q = &g->projs[q];
                    if (Q->d.post != p) continue;
                    double Eq = P->d.E_syn[Q->d.channel];
                    nu[g->g_off[q] + i] = aI * Q->scale * (Eq - V0[k]);      /* dL / dG_q[i] */
                    grad_scale[q] += aI * (Eq - V0[k]) * G[g->g_off[q] + i];
                }
            }
        }
        /* synapses: dL/dw_ik += r_i nu_k; pre gather into dL/dV_i */
        for (int q = 0; q < g->n_projs; ++q) {
            const gproj* Q = &g->projs[q];
            const gpop* pre = &g->pops[Q->d.pre];
            const double* nq = nu + g->g_off[q];
            for (int i = 0; i < pre->d.n; ++i) {
                double v = V0[pre->off + i];
                double r = release(v, Q->d.v_thr, Q->d.v_slope);
                double dr = r * (1.0 - r) / Q->d.v_slope;
                double acc = 0.0;
                for (int64_t e = Q->row_ptr[i]; e < Q->row_ptr[i + 1]; ++e) {
                    grad_w[q][e] += r * nq[Q->col[e]];
                    acc += Q->w[e] * nq[Q->col[e]];
                }
                nV[pre->off + i] += dr * acc;
            }
        }
        memcpy(lV, nV, (size_t)N * sizeof(double));
    }
    free(lV); free(lm); free(lh); free(ln); free(ly); free(nV); free(mu); free(nu); free(ie_now);
    return 0;
}

int oracle_graded_backward(graded_net* g, double* grad_scale, double** grad_w)
{
    return graded_backward(g, NULL, grad_scale, grad_w);
}

/* The adjoint seeded by the caller's dL/dy (T * N_out values, step-major). */
int oracle_graded_backward_dy(graded_net* g, const double* dL_dy, double* grad_scale, double** grad_w)
{
    if (!dL_dy) return -1;
    return graded_backward(g, dL_dy, grad_scale, grad_w);
}
